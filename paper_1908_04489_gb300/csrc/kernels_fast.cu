// kernels_fast.cu -- the fast path of the sweep (precision = 1).
//
// u0 step.  With E_m = U^(y_m) - y_m on the (extended) y grid, a candidate u
// whose positions u + w_l fall at y-index jb + l + t (exact integer jb,
// dyadic t) has  u - U^(u + w_l) = -(w_l + (1-t) E_{jb+l} + t E_{jb+l+1}),
// so the w quadrature S(u) of Section V-A's objective expands into three
// correlations of E against the fixed Gaussian weights:
//   S = W2 + 2[(1-t) P_p + t P_{p+1}] + (1-t)^2 Q_p + 2t(1-t) R_p + t^2 Q_{p+1},
//   W2 = sum phi_l w_l^2,  P_p = sum phi_l w_l E_{p+l},
//   Q_p = sum phi_l E_{p+l}^2,  R_p = sum phi_l E_{p+l} E_{p+l+1}.
// One table build per u1 update makes every candidate O(1).  The table value
// differs from the serial quadrature only by rounding; a bound on that
// difference screens each stage of the candidate list (Corollary 1's
// pointwise argmin, eq. (2)'s neighbour set, the coarse set and the
// refinement levels), and whenever two distinct values could still be the
// first minimum, those values are re-costed by the serial FP64 quadrature
// (kernels_plain.cu's arithmetic), so the winners are the plain path's.
//
// u1 step.  U_j = E[x1 | y1 = y_j] (Newton on the quadratic C_1, Section
// III-D; closed form of Section IV-C).  Along the uniform y grid the Gaussian
// weight of a source obeys w_{j+1} = w_j rho_j, rho_{j+1} = rho_j e^{-delta^2},
// so one exp per (source, run of 16 targets) replaces sixteen.  Pairs whose
// exponent exceeds the run's minimum by more than 46 (weight below 1e-20 of
// the largest) are skipped.
#include <float.h>
#include <limits.h>

#include "ucp_fast.cuh"

namespace ucp {

namespace {

constexpr int kRun = 16;          // targets per thread in the u1 recurrence
constexpr double kCut = 46.0;     // skip weights below e^-46 of the maximum

__device__ __forceinline__ double inv_one(const Geom& g) {
    return __longlong_as_double((int64_t)(1023 - g.shift) << 52);
}
__device__ __forceinline__ double value_of(const Geom& g, int64_t nu) {
    return __dmul_rn(__dmul_rn((double)nu, g.delta), inv_one(g));
}
__device__ __forceinline__ double x_of(const Geom& g, int64_t i) {
    return __dmul_rn((double)(i - g.hx), g.delta);
}

// Serial FP64 quadrature, operation for operation the plain path's S.
__device__ double S_exact(const Geom& g, const double* __restrict__ phi,
                          const double* __restrict__ U,
                          const double* __restrict__ Ud, int64_t nu) {
    const int64_t cell = nu >> g.shift;
    const double t = __dmul_rn((double)(nu - cell * g.one), inv_one(g));
    const int64_t jb = cell - g.hw + g.hy;
    const double u = value_of(g, nu);
    const int64_t ny1 = g.n_y - 1;
    double acc = 0.0;
    int64_t l = 0;
    const double eL = __dsub_rn(u, __dadd_rn(U[0], __dmul_rn(t, 0.0)));
    const double eL2 = __dmul_rn(eL, eL);
    for (; l < g.n_w && jb + l < 0; ++l)
        acc = __dadd_rn(acc, __dmul_rn(phi[l], eL2));
    for (; l < g.n_w && jb + l < ny1; ++l) {
        const int64_t j = jb + l;
        const double uh = __dadd_rn(U[j], __dmul_rn(t, Ud[j]));
        const double e = __dsub_rn(u, uh);
        acc = __dadd_rn(acc, __dmul_rn(phi[l], __dmul_rn(e, e)));
    }
    const double eR = __dsub_rn(u, __dadd_rn(U[ny1], __dmul_rn(t, 0.0)));
    const double eR2 = __dmul_rn(eR, eR);
    for (; l < g.n_w; ++l) acc = __dadd_rn(acc, __dmul_rn(phi[l], eR2));
    return acc;
}

__device__ __forceinline__ double control_term(const Geom& g, int64_t i,
                                               int64_t nu) {
    const double a = __dsub_rn(value_of(g, nu), x_of(g, i));
    return __dmul_rn(g.kk, __dmul_rn(a, a));
}

struct Eval {
    double gv;    // cost (table value or exact)
    double beta;  // bound on |gv - exact serial cost|, 0 when exact
};

// Cost of candidate nu at x_i from the correlation tables, with the bound.
__device__ __forceinline__ Eval eval_table(const Geom& g, const FastView& f,
                                           int64_t i, int64_t nu) {
    const int64_t cell = nu >> g.shift;
    const int64_t p = cell - f.c_lo;
    const double ctl = control_term(g, i, nu);
    if (p < 0 || p + 1 >= f.n_pos) {
        const double S = S_exact(g, f.phi, f.U, f.Ud, nu);
        return {__dadd_rn(ctl, S), 0.0};
    }
    const double t = __dmul_rn((double)(nu - cell * g.one), inv_one(g));
    const double omt = 1.0 - t;
    const double P0 = f.P[p], P1 = f.P[p + 1];
    const double Q0 = f.Q[p], Q1 = f.Q[p + 1];
    const double R0 = f.R[p];
    double S = f.W2 + 2.0 * (omt * P0 + t * P1) + omt * omt * Q0 +
               2.0 * t * omt * R0 + t * t * Q1;
    // M bounds the sum of the absolute values of every term (Cauchy-Schwarz:
    // |P_p| <= sqrt(W2 Q_p), |R_p| <= sqrt(Q_p Q_{p+1})).
    const float rm = sqrtf((float)f.W2) + (float)omt * sqrtf(fmaxf((float)Q0, 0.f)) +
                     (float)t * sqrtf(fmaxf((float)Q1, 0.f));
    const double M = (double)rm * (double)rm * (1.0 + 1e-5);
    const double gv = ctl + S;
    const double beta = f.beta_rel * M + f.beta_abs * (2.0 * (double)rm + 1.0) +
                        2.3e-16 * fabs(gv);
    return {gv, beta};
}

__device__ __forceinline__ double exact_cost(const Geom& g, const FastView& f,
                                             int64_t i, int64_t nu) {
    return __dadd_rn(control_term(g, i, nu), S_exact(g, f.phi, f.U, f.Ud, nu));
}

__device__ __forceinline__ bool before(double ga, int32_t pa, double gb,
                                       int32_t pb) {
    return ga < gb || (ga == gb && pa < pb);
}

template <int G>
__device__ __forceinline__ double gmin(double v) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
        v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off, G));
    return v;
}
template <int G>
__device__ __forceinline__ int64_t gmin_i64(int64_t v) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const int64_t o = __shfl_xor_sync(0xffffffffu, v, off, G);
        v = o < v ? o : v;
    }
    return v;
}
template <int G>
__device__ __forceinline__ int64_t gmax_i64(int64_t v) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const int64_t o = __shfl_xor_sync(0xffffffffu, v, off, G);
        v = o > v ? o : v;
    }
    return v;
}
template <int G>
__device__ __forceinline__ void glex(double& gv, int32_t& pos, int64_t& nu) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const double go = __shfl_xor_sync(0xffffffffu, gv, off, G);
        const int32_t po = __shfl_xor_sync(0xffffffffu, pos, off, G);
        const int64_t no = __shfl_xor_sync(0xffffffffu, nu, off, G);
        if (before(go, po, gv, pos)) { gv = go; pos = po; nu = no; }
    }
}

// The running winner: its value interval [gv - beta, gv + beta].
struct Best {
    double gv, beta;
    int32_t pos;
    int64_t nu;
};

// Candidate position p of stage 0 (incumbent, neighbours, coarse).
__device__ __forceinline__ int64_t stage0_nu(const Geom& g, const int64_t* nu_pre,
                                             const int64_t* coarse, int64_t i,
                                             int p) {
    if (p == 0) return nu_pre[i];
    if (p <= 2 * g.n_nbr) {
        const int d = p <= g.n_nbr ? p - g.n_nbr - 1 : p - g.n_nbr;
        int64_t ii = i + d;
        if (ii < 0 || ii >= g.n_x) ii = i;
        return nu_pre[ii];
    }
    return coarse[p - 1 - 2 * g.n_nbr];
}

// Resolve one stage: the candidates are the carried winner `best` (owned by
// lane 0) plus, for each lane, positions p0 + lane + k*G (k < per_lane) that
// are < p_end; cand(p) gives the lattice value.  Returns the first minimum
// of the exact serial costs over all of them, re-costing exactly only when
// the screened intervals leave more than one distinct value in play.
template <int G, typename CandFn>
__device__ Best resolve(const Geom& g, const FastView& f, int64_t i, int lane,
                        Best best, int p0, int p_end, CandFn cand,
                        int32_t* n_exact) {
    // 1. smallest upper end among all candidates
    double hi = lane == 0 ? best.gv + best.beta : DBL_MAX;
    for (int p = p0 + lane; p < p_end; p += G) {
        const Eval e = eval_table(g, f, i, cand(p));
        hi = fmin(hi, e.gv + e.beta);
    }
    hi = gmin<G>(hi);
    // 2. which distinct values can still be the minimum
    int64_t vmin = INT64_MAX, vmax = INT64_MIN;
    double tg = DBL_MAX;        // table value of the candidates in play
    int32_t tp = INT_MAX;
    int64_t tn = 0;
    if (lane == 0 && best.gv - best.beta <= hi) {
        vmin = vmax = best.nu;
        tg = best.gv; tp = best.pos; tn = best.nu;
    }
    for (int p = p0 + lane; p < p_end; p += G) {
        const int64_t nu = cand(p);
        const Eval e = eval_table(g, f, i, nu);
        if (e.gv - e.beta <= hi) {
            vmin = nu < vmin ? nu : vmin;
            vmax = nu > vmax ? nu : vmax;
            if (before(e.gv, p, tg, tp)) { tg = e.gv; tp = p; tn = nu; }
        }
    }
    vmin = gmin_i64<G>(vmin);
    vmax = gmax_i64<G>(vmax);
    if (vmin == vmax) {
        // one value in play: its first position wins; equal values carry
        // identical table costs, so the table-order first minimum is it
        glex<G>(tg, tp, tn);
        double beta = 0.0;
        if (tp == best.pos) beta = best.beta;
        else {
            const Eval e = eval_table(g, f, i, tn);
            beta = e.beta;
        }
        return {tg, beta, tp, tn};
    }
    // 3. several values in play: serial FP64 costs decide among them
    double xg = DBL_MAX;
    int32_t xp = INT_MAX;
    int64_t xn = 0;
    if (lane == 0 && best.gv - best.beta <= hi) {
        const double v = best.beta == 0.0 ? best.gv : exact_cost(g, f, i, best.nu);
        xg = v; xp = best.pos; xn = best.nu;
        if (best.beta != 0.0 && n_exact) atomicAdd(n_exact, 1);
    }
    for (int p = p0 + lane; p < p_end; p += G) {
        const int64_t nu = cand(p);
        const Eval e = eval_table(g, f, i, nu);
        if (e.gv - e.beta <= hi) {
            const double v = e.beta == 0.0 ? e.gv : exact_cost(g, f, i, nu);
            if (e.beta != 0.0 && n_exact) atomicAdd(n_exact, 1);
            if (before(v, p, xg, xp)) { xg = v; xp = p; xn = nu; }
        }
    }
    glex<G>(xg, xp, xn);
    return {xg, 0.0, xp, xn};
}

template <int G>
__global__ void __launch_bounds__(256) k_search_fast(Geom g, FastView f,
                                                     const int64_t* __restrict__ nu_pre,
                                                     int64_t* __restrict__ nu_out,
                                                     int32_t* __restrict__ idx_out,
                                                     int32_t* n_exact) {
    const int lane = threadIdx.x & (G - 1);
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const bool active = i < g.n_x;
    const int64_t ic = active ? i : g.n_x - 1;
    const int64_t* coarse = f.coarse;

    Best best{DBL_MAX, 0.0, INT_MAX, 0};
    const int n0 = 1 + 2 * g.n_nbr + g.n_coarse;
    best = resolve<G>(g, f, ic, lane, best, 0, n0,
                      [&](int p) { return stage0_nu(g, nu_pre, coarse, ic, p); },
                      active ? n_exact : nullptr);
    const int half = G / 2;
    int pos = n0;
    for (int lv = 1; lv <= g.n_levels; ++lv) {
        const int64_t h = g.q << (g.bits * (g.n_levels - lv));
        const int64_t centre = best.nu;
        best = resolve<G>(g, f, ic, lane, best, pos, pos + G,
                          [&](int p) {
                              const int k = p - pos;
                              const int64_t m = k < half ? k - half : k - half + 1;
                              return centre + m * h;
                          },
                          active ? n_exact : nullptr);
        pos += G;
    }
    if (active && lane == 0) {
        nu_out[i] = best.nu;
        idx_out[i] = best.pos;
    }
}

// ---- correlation tables -------------------------------------------------

// E_m = U^(y_m) - y_m for table E-index m (y-index jlo + m, U held constant
// beyond the table), its square, and E_m E_{m+1}; also Ud for exact costs.
__global__ void k_build_E(Geom g, FastView f, const double* __restrict__ U,
                          double* __restrict__ Ud) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < g.n_y) Ud[m] = m + 1 < g.n_y ? __dsub_rn(U[m + 1], U[m]) : 0.0;
    if (m >= f.n_e) return;
    const int64_t jj = f.jlo + m;
    const int64_t a = jj < 0 ? 0 : (jj > g.n_y - 1 ? g.n_y - 1 : jj);
    const int64_t b = jj + 1 < 0 ? 0 : (jj + 1 > g.n_y - 1 ? g.n_y - 1 : jj + 1);
    const double e0 = U[a] - (double)(jj - g.hy) * g.delta;
    const double e1 = U[b] - (double)(jj + 1 - g.hy) * g.delta;
    f.E[m] = e0;
    f.E2[m] = e0 * e0;
    f.EE[m] = e0 * e1;
}

constexpr int kTabT = 256;    // positions per block
constexpr int kTabL = 1024;   // taps per shared-memory chunk

__global__ void __launch_bounds__(kTabT) k_tables(Geom g, FastView f) {
    __shared__ double sE[kTabT + kTabL], sE2[kTabT + kTabL], sEE[kTabT + kTabL];
    __shared__ double sa[kTabL], sphi[kTabL];
    const int64_t p0 = (int64_t)blockIdx.x * kTabT;
    const int t = threadIdx.x;
    double P = 0.0, Q = 0.0, R = 0.0;
    for (int64_t l0 = 0; l0 < g.n_w; l0 += kTabL) {
        const int cl = (int)min((int64_t)kTabL, g.n_w - l0);
        __syncthreads();
        for (int k = t; k < kTabT + cl; k += kTabT) {
            const int64_t m = p0 + l0 + k;
            const bool ok = m < f.n_e;
            sE[k] = ok ? f.E[m] : 0.0;
            sE2[k] = ok ? f.E2[m] : 0.0;
            sEE[k] = ok ? f.EE[m] : 0.0;
        }
        for (int k = t; k < cl; k += kTabT) {
            sa[k] = f.a[l0 + k];
            sphi[k] = f.phi[l0 + k];
        }
        __syncthreads();
#pragma unroll 4
        for (int l = 0; l < cl; ++l) {
            P = fma(sa[l], sE[t + l], P);
            Q = fma(sphi[l], sE2[t + l], Q);
            R = fma(sphi[l], sEE[t + l], R);
        }
    }
    const int64_t p = p0 + t;
    if (p < f.n_pos) {
        f.P[p] = P;
        f.Q[p] = Q;
        f.R[p] = R;
    }
}

// a_l = phi_l w_l, W2 = sum phi_l w_l^2 (serial), prior_i = x_i^2 / 2 sigma^2,
// Yfac_j = exp(-delta y_j - delta^2 / 2).
__global__ void k_fast_setup(Geom g, FastView f) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < g.n_w) {
        const double w = (double)(k - g.hw) * g.delta;
        f.a[k] = f.phi[k] * w;
    }
    if (k < g.n_x) {
        const double x = x_of(g, k);
        f.prior[k] = __ddiv_rn(__dmul_rn(x, x), g.two_s2);
    }
    if (k < g.n_y) {
        const double y = (double)(k - g.hy) * g.delta;
        f.Yfac[k] = exp(-g.delta * y - 0.5 * g.delta * g.delta);
    }
    if (k == 0) {
        double s = 0.0;
        for (int64_t l = 0; l < g.n_w; ++l) {
            const double w = (double)(l - g.hw) * g.delta;
            s += f.phi[l] * (w * w);
        }
        *f.W2_dev = s;
    }
}

// ---- u1 step --------------------------------------------------------------

// Per source: f_i and exp(delta f_i) for this sweep.
__global__ void k_sources(Geom g, FastView f, const int64_t* __restrict__ nu) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_x) return;
    const double v = value_of(g, nu[i]);
    f.src_f[i] = v;
    f.src_F[i] = exp(g.delta * v);
}

// Approximate exponent minimum per target (FP32; only sets the scale).
constexpr int kShiftCh = 1024;
__global__ void __launch_bounds__(256) k_mmse_shift(Geom g, FastView f) {
    __shared__ float sp[kShiftCh], sf[kShiftCh];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float y = (float)((double)((j < g.n_y ? j : g.n_y - 1) - g.hy) * g.delta);
    float m = FLT_MAX;
    for (int64_t b = 0; b < g.n_x; b += kShiftCh) {
        const int cnt = (int)min((int64_t)kShiftCh, g.n_x - b);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            sp[k] = (float)f.prior[b + k];
            sf[k] = (float)f.src_f[b + k];
        }
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const float d = y - sf[k];
            m = fminf(m, fmaf(0.5f * d, d, sp[k]));
        }
    }
    if (j < g.n_y) f.mshift[j] = m;
}

constexpr int kMmseThreads = 64;
constexpr int kMmseSrc = 256;   // sources staged in shared memory at a time

__global__ void __launch_bounds__(kMmseThreads) k_mmse_main(Geom g, FastView f) {
    __shared__ double sf[kMmseSrc], sp[kMmseSrc], sF[kMmseSrc];
    const int64_t j0 = ((int64_t)blockIdx.x * kMmseThreads + threadIdx.x) * kRun;
    const int64_t c0 = (int64_t)blockIdx.y * f.chunk;
    const int64_t c1 = min(c0 + f.chunk, g.n_x);
    // shift of the run and its spread
    float smin = FLT_MAX, smax = -FLT_MAX;
    for (int k = 0; k < kRun; ++k) {
        const int64_t j = j0 + k < g.n_y ? j0 + k : g.n_y - 1;
        const float m = f.mshift[j];
        smin = fminf(smin, m);
        smax = fmaxf(smax, m);
    }
    const double srun = (double)smin;
    const double ya = (double)(j0 - g.hy) * g.delta;
    const double yb = (double)(j0 + kRun - 1 - g.hy) * g.delta;
    const double rho0 = f.Yfac[j0 < g.n_y ? j0 : g.n_y - 1];
    const double cstep = f.cstep;
    const float cut = (float)kCut + smax;
    double N[kRun], D[kRun];
#pragma unroll
    for (int k = 0; k < kRun; ++k) { N[k] = 0.0; D[k] = 0.0; }
    for (int64_t b = c0; b < c1; b += kMmseSrc) {
        const int cnt = (int)min((int64_t)kMmseSrc, c1 - b);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kMmseThreads) {
            sf[k] = f.src_f[b + k];
            sp[k] = f.prior[b + k];
            sF[k] = f.src_F[b + k];
        }
        __syncthreads();
        for (int s = 0; s < cnt; ++s) {
            const double fv = sf[s];
            const double pr = sp[s];
            const float dmin = fmaxf(0.f, fmaxf((float)(ya - fv), (float)(fv - yb)));
            if (fmaf(0.5f * dmin, dmin, (float)pr) - 1e-3f > cut) continue;
            const double d0 = ya - fv;
            double w = exp(srun - (pr + 0.5 * d0 * d0));
            double rho = rho0 * sF[s];
#pragma unroll
            for (int k = 0; k < kRun; ++k) {
                N[k] = fma(w, fv, N[k]);
                D[k] += w;
                w *= rho;
                rho *= cstep;
            }
        }
    }
    double* pN = f.partN + (size_t)blockIdx.y * g.n_y;
    double* pD = f.partD + (size_t)blockIdx.y * g.n_y;
#pragma unroll
    for (int k = 0; k < kRun; ++k)
        if (j0 + k < g.n_y) { pN[j0 + k] = N[k]; pD[j0 + k] = D[k]; }
}

__global__ void k_mmse_combine(Geom g, FastView f, double* __restrict__ U) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n_y) return;
    double n = 0.0, d = 0.0;
    for (int c = 0; c < f.n_chunks; ++c) {
        n += f.partN[(size_t)c * g.n_y + j];
        d += f.partD[(size_t)c * g.n_y + j];
    }
    U[j] = n / d;
}

// ---- J --------------------------------------------------------------------

constexpr int kJThreads = 256;
__global__ void __launch_bounds__(kJThreads) k_J_partial(Geom g, FastView f,
                                                         const double* __restrict__ px,
                                                         const int64_t* __restrict__ nu) {
    __shared__ double red[kJThreads];
    const int64_t i = (int64_t)blockIdx.x * kJThreads + threadIdx.x;
    double v = 0.0;
    if (i < g.n_x) v = px[i] * eval_table(g, f, i, nu[i]).gv;
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = kJThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) f.Jpart[blockIdx.x] = red[0];
}

__global__ void k_J_final(FastView f, int nblk, double* out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += f.Jpart[b];
    *out = s;
}

inline unsigned blocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// ---- host-side plan and launches ------------------------------------------

void fast_plan(const Geom& g, FastPlan* fp) {
    // cells reachable by any candidate: coarse extremes plus the refinement
    // reach (< 1.15 q), or the x0 range (identity init), with margin
    const int64_t reach = (int64_t)(g.n_coarse - 1) * (g.q / 2) + 2 * g.q;
    const int64_t ext = (reach > g.hx + 2 * g.q ? reach : g.hx + 2 * g.q) + 2;
    fp->c_lo = -ext;
    fp->n_pos = 2 * ext + 2;
    fp->jlo = fp->c_lo - g.hw + g.hy;
    fp->n_e = fp->n_pos + g.n_w + 1;
    const int64_t jblocks = (g.n_y + kMmseThreads * kRun - 1) / (kMmseThreads * kRun);
    int64_t chunks = (4 * 152 + jblocks - 1) / jblocks;
    const int64_t max_chunks = (g.n_x + 127) / 128;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    const int64_t chunk = ((g.n_x + chunks - 1) / chunks + 63) / 64 * 64;
    fp->chunk = chunk;
    fp->n_chunks = (int)((g.n_x + chunk - 1) / chunk);
    fp->j_blocks = jblocks;
    fp->J_blocks = (g.n_x + kJThreads - 1) / kJThreads;
}

void launch_fast_setup(const Geom& g, const FastView& f, cudaStream_t s) {
    int64_t n = g.n_w > g.n_x ? g.n_w : g.n_x;
    n = n > g.n_y ? n : g.n_y;
    k_fast_setup<<<blocks(n, 256), 256, 0, s>>>(g, f);
}

void launch_mmse_fast(const Geom& g, const FastView& f, const int64_t* nu,
                      double* U, cudaStream_t s, Prof* prof) {
    cudaEvent_t ev;
    int k = prof ? prof->begin("mmse_sources", &ev) : -1;
    k_sources<<<blocks(g.n_x, 256), 256, 0, s>>>(g, f, nu);
    if (prof) prof->end(k, ev);
    k = prof ? prof->begin("mmse_shift", &ev) : -1;
    k_mmse_shift<<<blocks(g.n_y, 256), 256, 0, s>>>(g, f);
    if (prof) prof->end(k, ev);
    k = prof ? prof->begin("mmse_main", &ev) : -1;
    dim3 grid((unsigned)f.j_blocks, (unsigned)f.n_chunks);
    k_mmse_main<<<grid, kMmseThreads, 0, s>>>(g, f);
    if (prof) prof->end(k, ev);
    k = prof ? prof->begin("mmse_combine", &ev) : -1;
    k_mmse_combine<<<blocks(g.n_y, 256), 256, 0, s>>>(g, f, U);
    if (prof) prof->end(k, ev);
}

void launch_tables(const Geom& g, const FastView& f, const double* U, double* Ud,
                   cudaStream_t s, Prof* prof) {
    cudaEvent_t ev;
    const int64_t n = f.n_e > g.n_y ? f.n_e : g.n_y;
    int k = prof ? prof->begin("build_E", &ev) : -1;
    k_build_E<<<blocks(n, 256), 256, 0, s>>>(g, f, U, Ud);
    if (prof) prof->end(k, ev);
    k = prof ? prof->begin("tables", &ev) : -1;
    k_tables<<<blocks(f.n_pos, kTabT), kTabT, 0, s>>>(g, f);
    if (prof) prof->end(k, ev);
}

void launch_search_fast(const Geom& g, const FastView& f, const int64_t* nu_in,
                        int64_t* nu_out, int32_t* idx, cudaStream_t s) {
    const int64_t threads = g.n_x * (int64_t)g.n_refine;
    const int bs = 256;
#define UCP_FAST_CASE(G)                                                   \
    case G:                                                                \
        k_search_fast<G><<<blocks(threads, bs), bs, 0, s>>>(g, f, nu_in,   \
                                                          nu_out, idx,     \
                                                          f.n_exact);      \
        break;
    switch (g.n_refine) {
        UCP_FAST_CASE(2)
        UCP_FAST_CASE(4)
        UCP_FAST_CASE(8)
        UCP_FAST_CASE(16)
        UCP_FAST_CASE(32)
        default: break;
    }
#undef UCP_FAST_CASE
}

void launch_J_fast(const Geom& g, const FastView& f, const double* px,
                   const int64_t* nu, double* out, cudaStream_t s, Prof* prof) {
    cudaEvent_t ev;
    int k = prof ? prof->begin("J_partial", &ev) : -1;
    k_J_partial<<<(unsigned)f.J_blocks, kJThreads, 0, s>>>(g, f, px, nu);
    if (prof) prof->end(k, ev);
    k = prof ? prof->begin("J_final", &ev) : -1;
    k_J_final<<<1, 32, 0, s>>>(f, (int)f.J_blocks, out);
    if (prof) prof->end(k, ev);
}

}  // namespace ucp
