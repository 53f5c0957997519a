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
// One table build per u1 update (on the tensor cores, kernels_tc.cu) makes
// every candidate O(1).  A table cost
// differs from the serial FP64 quadrature only by rounding; a rigorous bound
// on that difference screens each stage of the candidate list (Corollary 1's
// pointwise argmin over eq. (2)'s neighbours, the coarse set and the
// refinement levels).  Whenever two distinct values could still be the first
// minimum, those values are re-costed by the serial FP64 quadrature (the
// plain path's arithmetic, operation for operation), so the fast path makes
// the plain path's decisions.
//
// The u1 step (U_j = E[x1 | y1 = y_j]) is in kernels_u1.cu.
//
// Arithmetic: the screening runs in double-float on the FP32 pipe (df.cuh);
// FP64 only combines partial sums and re-costs near-ties.
#include <float.h>
#include <limits.h>

#include <algorithm>

#include "df.cuh"
#include "fixed_sum.cuh"
#include "ucp_fast.cuh"

namespace ucp {

namespace {


__device__ __forceinline__ double inv_one(const Geom& g) {
    return __longlong_as_double((int64_t)(1023 - g.shift) << 52);
}
__device__ __forceinline__ double value_of(const Geom& g, int64_t nu) {
    return __dmul_rn(__dmul_rn((double)nu, g.delta), inv_one(g));
}
__device__ __forceinline__ double x_of(const Geom& g, int64_t i) {
    return __dmul_rn((double)(i - g.hx), g.delta);
}

// ---- exact serial FP64 cost (the plain path's arithmetic) -----------------

__device__ __forceinline__ double exact_term(const Geom& g,
                                             const double* __restrict__ phi,
                                             const double* __restrict__ U,
                                             const double* __restrict__ Ud,
                                             int64_t jb, double t, double u,
                                             int64_t l) {
    const int64_t j = jb + l;
    double uh;
    if (j < 0) uh = __dadd_rn(U[0], __dmul_rn(t, 0.0));
    else if (j >= g.n_y - 1) uh = __dadd_rn(U[g.n_y - 1], __dmul_rn(t, 0.0));
    else uh = __dadd_rn(U[j], __dmul_rn(t, Ud[j]));
    const double e = __dsub_rn(u, uh);
    return __dmul_rn(phi[l], __dmul_rn(e, e));
}

template <int G>
__device__ __forceinline__ unsigned group_mask();

// single-lane variant (rare: candidates outside the table range)
__device__ double exact_cost_lane(const Geom& g, const FastView& f, int64_t i,
                                  int64_t nu) {
    const int64_t cell = nu >> g.shift;
    const double t = __dmul_rn((double)(nu - cell * g.one), inv_one(g));
    const int64_t jb = cell - g.hw + g.hy;
    const double u = value_of(g, nu);
    FixedSum acc;
    for (int64_t l = 0; l < g.n_w; ++l) acc.add(exact_term(g, f.phi, f.U, f.Ud, jb, t, u, l));
    const double a = __dsub_rn(u, x_of(g, i));
    return __dadd_rn(__dmul_rn(g.kk, __dmul_rn(a, a)), acc.result());
}

constexpr int kTieBatch = 8;   // candidates re-costed exactly per pass

// Second screening tier: the direct w quadrature of S from the E table,
// taps split over the group.  The residual
//   d_l = (w_l + E_{p+l}) + t (E_{p+l+1} - E_{p+l})
// is formed with accurate double-float additions (error relative to the
// small results, not to the operands), each term phi_l d_l^2 in double-float,
// 8-term double-float blocks summed in FP64 and reduced over the lanes in a
// fixed order (every lane gets the same value).  The sum has no cancellation, so its
// bound is several times tighter than the table identity's.  Candidates
// outside the tables get an infinite bound (no second tier).
// Shared state of the block-cooperative tiers: cross-group partial sums of
// the second tier, the members and results of the exact costs, and the
// block's scratch (the groups' shared columns, free once screening is done).
constexpr int kCoopT = 256;   // threads per block of the deferred search
// additions per thread in one level of the exact costs' chunk tree: a level
// of mb candidates holds at most mb * nch / 2 <= kCoopT * kTieBatch / 2 pairs
constexpr int kTreeAdds = kTieBatch / 2;
static_assert(kTreeAdds * 2 == kTieBatch, "tree additions per thread");
struct CoopSmem {
    double acc[kCoopT / 2][2];
    float emax[kCoopT / 2][2], demax[kCoopT / 2][2];
    double res2[2][2];   // second-tier cost and bound of the two candidates
    int64_t mem_nu[32];
    double res[32];
    double* scratch;   // kCoopT * kTieBatch doubles
};

// Exact FP64 costs (the plain path's arithmetic, terms summed in the fixed
// order of fixed_sum.cuh) of the M <= 32 candidates held in lanes m < M of
// every group; all groups of the block call this with the same candidates.
// The block forms the chunk sums of all candidates in parallel, then thread
// m merges candidate m's chunks in order.  Valid in lanes < M.
template <int G>
__device__ double exact_costs_coop(const Geom& g, const FastView& f, int64_t i,
                                   int lane, int64_t nu, int M, CoopSmem* cs) {
    __syncthreads();   // every group is done with its scratch column
    if (threadIdx.x < (unsigned)M) cs->mem_nu[threadIdx.x] = nu;   // group 0's lanes
    __syncthreads();
    const int64_t nch = sum_chunks(g.n_w);
    const int64_t cap = (int64_t)kCoopT * kTieBatch;
    double* ch = cs->scratch;
    const int per = (int)max((int64_t)1, min((int64_t)M, cap / nch));
    // chunk k of candidate m: terms 32k .. 32k + 31 added left to right
    auto chunk = [&](int64_t cnu, int64_t k) {
        const int64_t cell = cnu >> g.shift;
        const double t = __dmul_rn((double)(cnu - cell * g.one), inv_one(g));
        const int64_t jb = cell - g.hw + g.hy;
        const double u = value_of(g, cnu);
        const int64_t e = min((k + 1) * kSumChunk, g.n_w);
        double a = 0.0;
        int64_t l = k * kSumChunk;
        // eight terms as independent chains, then added in order
        for (; l + 8 <= e; l += 8) {
            double tm[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                tm[q] = exact_term(g, f.phi, f.U, f.Ud, jb, t, u, l + q);
#pragma unroll
            for (int q = 0; q < 8; ++q) a = __dadd_rn(a, tm[q]);
        }
        for (; l < e; ++l) a = __dadd_rn(a, exact_term(g, f.phi, f.U, f.Ud, jb, t, u, l));
        return a;
    };
    for (int m0 = 0; m0 < M; m0 += per) {
        const int mb = min(per, M - m0);
        if ((int64_t)mb * nch <= cap) {
            // every chunk sum of the mb candidates in shared memory, then the
            // fixed pairwise tree level by level, each level's additions in
            // parallel: entries (2k, 2k + 1) of a level give entry k of the
            // next, an unpaired last entry moving up unchanged (the order of
            // fixed_sum.cuh, so the same double)
            for (int64_t idx = threadIdx.x; idx < mb * nch; idx += blockDim.x) {
                const int m = (int)(idx / nch);
                ch[idx] = chunk(cs->mem_nu[m0 + m], idx % nch);
            }
            __syncthreads();
            for (int64_t n = nch; n > 1;) {
                const int64_t h = n / 2;    // mb * h <= cap / 2 = kTreeAdds * blockDim.x
                double v[kTreeAdds];
                int nv = 0;
                for (int64_t idx = threadIdx.x; idx < mb * h; idx += blockDim.x) {
                    const int64_t m = idx / h, k = idx % h;
                    v[nv++] = __dadd_rn(ch[m * nch + 2 * k], ch[m * nch + 2 * k + 1]);
                }
                double mv = 0.0;
                if ((n & 1) && threadIdx.x < (unsigned)mb) mv = ch[threadIdx.x * nch + n - 1];
                __syncthreads();
                nv = 0;
                for (int64_t idx = threadIdx.x; idx < mb * h; idx += blockDim.x) {
                    const int64_t m = idx / h, k = idx % h;
                    ch[m * nch + k] = v[nv++];
                }
                if ((n & 1) && threadIdx.x < (unsigned)mb) ch[threadIdx.x * nch + h] = mv;
                __syncthreads();
                n = h + (n & 1);
            }
            if (threadIdx.x < (unsigned)mb) {
                const int64_t cnu = cs->mem_nu[m0 + threadIdx.x];
                const double a = __dsub_rn(value_of(g, cnu), x_of(g, i));
                cs->res[m0 + threadIdx.x] =
                    __dadd_rn(__dmul_rn(g.kk, __dmul_rn(a, a)), ch[threadIdx.x * nch]);
            }
            __syncthreads();
            continue;
        }
        // one candidate with more chunks than the scratch holds: chunks in
        // passes, each pass's sums streamed into the binary-counter stack
        const int64_t span = cap;
        FixedSum acc;
        for (int64_t c0 = 0; c0 < nch; c0 += span) {
            const int64_t cn = min(span, nch - c0);
            for (int64_t idx = threadIdx.x; idx < cn; idx += blockDim.x)
                ch[idx] = chunk(cs->mem_nu[m0], c0 + idx);
            __syncthreads();
            if (threadIdx.x == 0)
                for (int64_t k = 0; k < cn; ++k) acc.push_chunk(ch[k]);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const int64_t cnu = cs->mem_nu[m0];
            const double a = __dsub_rn(value_of(g, cnu), x_of(g, i));
            cs->res[m0] = __dadd_rn(__dmul_rn(g.kk, __dmul_rn(a, a)), acc.result());
        }
    }
    __syncthreads();
    return lane < M ? cs->res[lane] : 0.0;
}

// With cs == nullptr the group's G lanes take every tap; otherwise the
// blockDim.x / G groups of the block (all costing the same candidates) split
// the taps and their partial sums are combined in group order.
template <int G>
__device__ void direct_df_cost2(const Geom& g, const FastView& f, int64_t i,
                                const int64_t (&nu)[2], int lane, double (&g2)[2],
                                double (&b2)[2], CoopSmem* cs = nullptr) {
    // two candidates per pass over the taps (independent chains interleave)
    const unsigned gm = group_mask<G>();
    const int part = cs ? (int)(threadIdx.x / G) : 0;
    const int nparts = cs ? (int)(blockDim.x / G) : 1;
    int64_t p[2];
    dfloat t[2];
    bool ok[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int64_t cell = nu[b] >> g.shift;
        p[b] = cell - f.c_lo;
        ok[b] = p[b] >= 0 && p[b] + 1 < f.n_pos;
        if (!ok[b]) p[b] = 0;
        t[b] = df_mul_f(df_from_i64(nu[b] - cell * g.one), f.inv_one_f);
    }
    double acc[2] = {0.0, 0.0};
    dfloat blk[2] = {{0.f, 0.f}, {0.f, 0.f}};
    float emax[2] = {0.f, 0.f}, demax[2] = {0.f, 0.f};
    int cnt = 0;
#pragma unroll 2
    for (int64_t l = part * G + lane; l < g.n_w; l += G * nparts) {
        const dfloat w = f.wdf[l], ph = f.phidf[l];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const dfloat E0 = f.E[p[b] + l], E1 = f.E[p[b] + l + 1];
            const dfloat dE = df_add_acc(E1, df_neg(E0));
            const dfloat d = df_add_acc(df_add_acc(w, E0), df_mul(t[b], dE));
            blk[b] = df_add(blk[b], df_mul(ph, df_mul(d, d)));
            emax[b] = fmaxf(emax[b], fmaxf(fabsf(E0.hi), fabsf(E1.hi)));
            demax[b] = fmaxf(demax[b], fabsf(dE.hi));
        }
        if (++cnt == 8) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                acc[b] += df_to_double(blk[b]);
                blk[b] = {0.f, 0.f};
            }
            cnt = 0;
        }
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        acc[b] += df_to_double(blk[b]);
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
            acc[b] += __shfl_down_sync(gm, acc[b], off, G);
            emax[b] = fmaxf(emax[b], __shfl_down_sync(gm, emax[b], off, G));
            demax[b] = fmaxf(demax[b], __shfl_down_sync(gm, demax[b], off, G));
        }
    }
    // cost and bound of candidate b from the combined sums (every lane of a
    // group, or one thread of the block, gets the same values).  The bound is
    // formed in FP32 from positive terms (at most ~12 roundings of 2^-24 each,
    // covered by the factor 1.00001); the cost stays FP64.
    auto finish = [&](int b, double S2, float em, float dm, double& gv, double& bv) {
        if (!ok[b]) {
            gv = 0.0;
            bv = INFINITY;
            return;
        }
        const dfloat a = df_mul(df_from_i64(nu[b] - (i - g.hx) * g.one),
                                dfloat{f.step_hi, f.step_lo});
        const dfloat ctl = df_mul(dfloat{f.kk_hi, f.kk_lo}, df_mul(a, a));
        const double c = df_to_double(ctl);
        gv = c + S2;
        // |error of d_l| <= uf^2 (|w_l| + |E_{p+l}| + |E_{p+l+1}|) from the
        // double-float representations plus 8 uf^2 (|d_l| + |dE_l|) from the
        // operations; summed against phi_l 2|d_l| this gives the terms below.
        const float uf2 = 0x1p-48f;
        const float s2 = fmaxf((float)S2, 0.0f) * 1.000001f;
        const float rs = sqrtf(s2) * 1.000001f;
        const float cf = fabsf(ctl.hi) * 1.000001f;
        const float eps = f.beta_abs + uf2 * (f.w_half + 2.0f * em);
        const float bf = f.beta2_rel * s2 + 1.25f * 16.0f * uf2 * (s2 + rs * dm) +
                         1.25f * (2.0f * rs + 1.0f) * eps + 3.0e-13f * cf +
                         f.beta_ctl * (f.k_f * fabsf(a.hi) * 1.0001f) +
                         4.0e-16f * (float)fabs(gv) * 1.000001f;
        bv = (double)(bf * 1.00001f);
    };
    if (cs) {
        // the groups' partials are reduced by warp 0 (a fixed tree) and the
        // tail runs once per candidate (lanes 0 and 1), shared through
        // shared memory
        if (lane == 0) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                cs->acc[part][b] = acc[b];
                cs->emax[part][b] = emax[b];
                cs->demax[part][b] = demax[b];
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int q = threadIdx.x;
            double S[2];
            float em[2], dm[2];
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                S[b] = q < nparts ? cs->acc[q][b] : 0.0;
                em[b] = q < nparts ? cs->emax[q][b] : 0.0f;
                dm[b] = q < nparts ? cs->demax[q][b] : 0.0f;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    S[b] += __shfl_down_sync(0xffffffffu, S[b], off);
                    em[b] = fmaxf(em[b], __shfl_down_sync(0xffffffffu, em[b], off));
                    dm[b] = fmaxf(dm[b], __shfl_down_sync(0xffffffffu, dm[b], off));
                }
            }
            const double S1 = __shfl_sync(0xffffffffu, S[1], 0);
            const float em1 = __shfl_sync(0xffffffffu, em[1], 0);
            const float dm1 = __shfl_sync(0xffffffffu, dm[1], 0);
            if (q == 0) finish(0, S[0], em[0], dm[0], cs->res2[0][0], cs->res2[0][1]);
            if (q == 1) finish(1, S1, em1, dm1, cs->res2[1][0], cs->res2[1][1]);
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            g2[b] = cs->res2[b][0];
            b2[b] = cs->res2[b][1];
        }
        __syncthreads();
        return;
    }
#pragma unroll
    for (int b = 0; b < 2; ++b)
        finish(b, __shfl_sync(gm, acc[b], 0, G), __shfl_sync(gm, emax[b], 0, G),
               __shfl_sync(gm, demax[b], 0, G), g2[b], b2[b]);
}

// ---- certified cost differences (between the second and third tiers) ------
//
// For two candidates r and m in one cell (fractions t_r, t_m = t_r + dt) the
// residuals differ by dt dE_l, so
//   S(m) - S(r) = sum_l phi_l dt dE_l (2 d_l(r) + dt dE_l),
// a sum of small terms (no cancellation against S), and the control terms
// differ by k^2 (u_m - u_r)(u_m + u_r - 2 x).  The block forms this in
// double-float with a bound e_est far below the FP64 rounding of either cost;
// the serial FP64 costs (the plain path's arithmetic on the same table) obey
// |g_o(x) - g(x)| <= err_o(x) = beta_rel S + 2u (B + 3D) sqrt(S) + the
// control term's and the final addition's roundings, B = max |U| and D =
// max |U_{j+1} - U_j| over the taps (each residual's rounding is below
// u (|e| + B + 3D), its square's below 3u e^2 + 2u |e| (B + 3D)).  When the
// estimated difference exceeds e_est + err_o(m) + err_o(r), m's serial cost
// is certainly above r's.  `delta` and `thresh` are the same in every thread.
template <int G>
__device__ void diff_df_coop(const Geom& g, const FastView& f, int64_t i, int64_t nu_r,
                             int64_t nu_m, int lane, CoopSmem* cs, double& delta,
                             double& thresh) {
    const unsigned gm = group_mask<G>();
    const int part = (int)(threadIdx.x / G), nparts = (int)(blockDim.x / G);
    const int64_t cell = nu_r >> g.shift, p = cell - f.c_lo;
    const dfloat t = df_mul_f(df_from_i64(nu_r - cell * g.one), f.inv_one_f);
    const dfloat dt = df_mul_f(df_from_i64(nu_m - nu_r), f.inv_one_f);
    // each thread's terms summed in double-float (off the FP64 pipe), then
    // the threads' sums in FP64
    dfloat bd{0.f, 0.f}, bs{0.f, 0.f};
    float t1 = 0.f, t3 = 0.f, emax = 0.f, demax = 0.f;
#pragma unroll 2
    for (int64_t l = part * G + lane; l < g.n_w; l += G * nparts) {
        const dfloat w = f.wdf[l], ph = f.phidf[l];
        const dfloat E0 = f.E[p + l], E1 = f.E[p + l + 1];
        const dfloat dE = df_add_acc(E1, df_neg(E0));
        const dfloat d = df_add_acc(df_add_acc(w, E0), df_mul(t, dE));
        const dfloat dd = df_mul(dt, dE);
        const dfloat s2 = df_add(df_add(d, d), dd);
        const dfloat term = df_mul(ph, df_mul(dd, s2));
        bd = df_add(bd, term);
        bs = df_add(bs, df_mul(ph, df_mul(d, d)));
        t1 = fmaf(ph.hi, fabsf(s2.hi), t1);
        t3 += fabsf(term.hi);
        emax = fmaxf(emax, fmaxf(fabsf(E0.hi), fabsf(E1.hi)));
        demax = fmaxf(demax, fabsf(dE.hi));
    }
    double acc_d = df_to_double(bd), acc_s = df_to_double(bs);
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        acc_d += __shfl_down_sync(gm, acc_d, off, G);
        acc_s += __shfl_down_sync(gm, acc_s, off, G);
        t1 += __shfl_down_sync(gm, t1, off, G);
        t3 += __shfl_down_sync(gm, t3, off, G);
        emax = fmaxf(emax, __shfl_down_sync(gm, emax, off, G));
        demax = fmaxf(demax, __shfl_down_sync(gm, demax, off, G));
    }
    __syncthreads();   // cs is free (the previous user has read its results)
    if (lane == 0) {
        cs->acc[part][0] = acc_d;
        cs->acc[part][1] = acc_s;
        cs->emax[part][0] = emax;
        cs->emax[part][1] = demax;
        cs->demax[part][0] = t1;
        cs->demax[part][1] = t3;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int q = threadIdx.x;
        double dS = q < nparts ? cs->acc[q][0] : 0.0, Sr = q < nparts ? cs->acc[q][1] : 0.0;
        float em = q < nparts ? cs->emax[q][0] : 0.f, dm = q < nparts ? cs->emax[q][1] : 0.f;
        float T1 = q < nparts ? cs->demax[q][0] : 0.f, T3 = q < nparts ? cs->demax[q][1] : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dS += __shfl_down_sync(0xffffffffu, dS, off);
            Sr += __shfl_down_sync(0xffffffffu, Sr, off);
            em = fmaxf(em, __shfl_down_sync(0xffffffffu, em, off));
            dm = fmaxf(dm, __shfl_down_sync(0xffffffffu, dm, off));
            T1 += __shfl_down_sync(0xffffffffu, T1, off);
            T3 += __shfl_down_sync(0xffffffffu, T3, off);
        }
        if (q == 0) {
            const double u = 0x1p-53, uf = 0x1p-48;
            const dfloat step{f.step_hi, f.step_lo}, kk{f.kk_hi, f.kk_lo};
            const int64_t base = (i - g.hx) * g.one, dnu = nu_m - nu_r;
            const int64_t snu = nu_m + nu_r - 2 * base;
            const int64_t lim = (int64_t)1 << 44;
            const dfloat dctl = df_mul(kk, df_mul(df_mul(df_from_i64(dnu), step),
                                                  df_mul(df_from_i64(snu), step)));
            const double dc = df_to_double(dctl);
            delta = dS + dc;
            // magnitudes (FP64, rounded up by the final factor)
            const double Y = (double)f.y_abs, B = (double)em + Y;
            const double D = (double)dm + (double)f.delta_hi * 1.0001;
            const double adt = fabs(df_to_double(dt));
            const double sr = fmax(Sr, 0.0) * 1.01 + 1e-300, sm = fmax(Sr + dS, 0.0) * 1.01 + 1e-300;
            auto err_o = [&](int64_t nu, double S) {
                const double a = fabs(df_to_double(df_mul(df_from_i64(nu - base), step)));
                const double uv = fabs(df_to_double(df_mul(df_from_i64(nu), step)));
                const double xv = fabs((double)(i - g.hx)) * (double)f.delta_hi;
                const double ctl = (double)f.kk_hi * a * a;
                return (double)f.beta_rel * S + 2.0 * u * (B + 3.0 * D) * sqrt(S) +
                       2.0 * u * (double)f.kk_hi * a * (uv + xv + 2.0 * a) + 4.0 * u * (ctl + S);
            };
            // the estimate's own error: the E table's representation (relative
            // 2^-48 of |E| + |y|) in dt dE and in the residuals, each term's
            // double-float operations (8 uf) and its thread's double-float sum
            // of K terms (2 uf per addition), the FP64 sums over the threads,
            // all below (K + 8) 2^-46 of the terms' magnitudes, and the control
            // difference (8 uf of itself)
            const double K = (double)((g.n_w + G * nparts - 1) / (G * nparts));
            const double epsE = 1.1 * uf * (B + Y);
            const double e_est = 1.25 * (2.0 * adt * epsE * (double)T1 +
                                         2.0 * uf * (f.w_half + 4.0 * B + dm) * adt * dm +
                                         (K + 8.0) * 0x1p-46 * (double)T3) +
                                 8.0 * uf * fabs(dc);
            const bool ok = llabs(snu) < lim && llabs(dnu) < lim;
            thresh = ok ? (e_est + err_o(nu_m, sm) + err_o(nu_r, sr)) * 1.01 + 1e-300
                        : INFINITY;
            cs->res2[0][0] = delta;
            cs->res2[0][1] = thresh;
        }
    }
    __syncthreads();
    delta = cs->res2[0][0];
    thresh = cs->res2[0][1];
    __syncthreads();
}

// ---- screened table cost ------------------------------------------------

struct Eval {
    dfloat gv;    // cost
    float beta;   // bound on |gv - serial FP64 cost|
};

// The table identity at cell p (positions p and p + 1) as a quadratic in the
// cell fraction t:
//   S = A0 + t (A1 + t A2),  A0 = W2 + 2 P_p + Q_p,
//   A1 = 2 (P_{p+1} - P_p) + 2 (R_p - Q_p),  A2 = Q_p + Q_{p+1} - 2 R_p,
// in double-float, and B, the cell's bound on |table S - serial FP64 S| at
// any t in [0, 1]: the tables' own error (tc_bt of the cell's columns), the
// serial path's rounding beta_rel M and beta_abs (2 sqrt(M) + 1) with
// M = (sqrt(W2) + max(sqrt(Q_p), sqrt(Q_{p+1})))^2, which bounds the sum of
// |terms| of the w quadrature (Cauchy-Schwarz), and the rounding of the
// quadratic itself from the actual magnitudes (double-float additions err by
// <= 2 u^2 (|a| + |b|), products by <= 5 u^2 |a b|, u = 2^-24; t is exact):
//   coefficients  2 (W2 + 4|P_p| + 2 Q_p) + 8 (|P_p| + |P_{p+1}| + |R_p| + Q_p)
//                 + 4 (Q_p + Q_{p+1} + |R_p|),
//   Horner and the sum with the control term
//                 5 |A2| + 7 (|A1| + |A2|) + 4 (|A0| + |A1| + |A2|),  times u^2.
struct Coef {
    dfloat a0, a1, a2;
    float b;
};

__device__ __forceinline__ dfloat df_x2(dfloat v) { return {2.0f * v.hi, 2.0f * v.lo}; }

// W2 = sum phi_l w_l^2 (set-up kernel's fixed-order sum, read from the
// device) as double-float, and sqrt(W2) rounded up by 1e-4 in FP32.
struct W2v {
    dfloat w;
    float sq;
};
__device__ __forceinline__ W2v w2_of(const FastView& f) {
    const double W2 = __ldg(f.W2_dev);
    return {df_from_double(W2), __fmul_rn(__double2float_rn(__dsqrt_rn(W2)), 1.0001f)};
}

__device__ __forceinline__ Coef coef_of(const FastView& f, int64_t p, const W2v& W2) {
    const dfloat P0 = f.P[p], P1 = f.P[p + 1];
    const dfloat Q0 = f.Q[p], Q1 = f.Q[p + 1];
    const dfloat R0 = f.R[p];
    Coef c;
    c.a0 = df_add(W2.w, df_add(df_x2(P0), Q0));
    c.a1 = df_add(df_add(df_x2(P1), df_neg(df_x2(P0))), df_add(df_x2(R0), df_neg(df_x2(Q0))));
    c.a2 = df_add(df_add(Q0, Q1), df_neg(df_x2(R0)));
    const float q0 = fmaxf(Q0.hi, 0.f), q1 = fmaxf(Q1.hi, 0.f);
    const float rm = (W2.sq + fmaxf(sqrtf(q0), sqrtf(q1))) * 1.0001f;
    const float M = rm * rm * 1.0001f;
    const int64_t a1 = p >> 7, a2 = (p + 1) >> 7;
    const float bt = f.tc_bt[a1] + (a2 != a1 ? f.tc_bt[a2] : 0.f);
    const float p0 = fabsf(P0.hi), p1 = fabsf(P1.hi), r0 = fabsf(R0.hi);
    const float b0 = fabsf(c.a0.hi), b1 = fabsf(c.a1.hi), b2 = fabsf(c.a2.hi);
    const float e_coef = 2.0f * (W2.w.hi + 4.0f * p0 + 2.0f * q0) +
                         8.0f * (p0 + p1 + r0 + q0) + 4.0f * (q0 + q1 + r0);
    const float e_eval = 5.0f * b2 + 7.0f * (b1 + b2) + 4.0f * (b0 + b1 + b2);
    c.b = (bt + f.beta_rel * M + f.beta_abs * (2.0f * rm + 1.0f) +
           1.25f * 1.01f * 0x1p-48f * (e_coef + e_eval)) * 1.0001f;
    return c;
}

// g(u; x_i) = k^2 (u - x_i)^2 + S from the cell's quadratic; the bound adds
// the control term's rounding (k |u - x_i| = sqrt of the control term).
__device__ __forceinline__ Eval eval_poly(const Geom& g, const FastView& f, int64_t i,
                                          int64_t nu, dfloat t, const Coef& c) {
    const dfloat S = df_add(c.a0, df_mul(t, df_add(c.a1, df_mul(t, c.a2))));
    const dfloat a = df_mul(df_from_i64(nu - (i - g.hx) * g.one), dfloat{f.step_hi, f.step_lo});
    const dfloat ctl = df_mul(dfloat{f.kk_hi, f.kk_lo}, df_mul(a, a));
    const dfloat gv = df_add(ctl, S);
    const float beta = c.b + 3.0e-13f * fabsf(ctl.hi) +
                       f.beta_ctl * (f.k_f * fabsf(a.hi) * 1.0001f) + 4.0e-16f * fabsf(gv.hi);
    return {gv, beta};
}

// Outside the tables (rare): the serial cost, the bound covering its rounding
// to double-float.
__device__ __forceinline__ Eval eval_outside(const Geom& g, const FastView& f, int64_t i,
                                             int64_t nu) {
    const double v = exact_cost_lane(g, f, i, nu);
    return {df_from_double(v), 4.0e-15f * (float)fabs(v) + FLT_MIN};
}

// Screened cost of candidate nu for x0 point i from the stored cell
// coefficients (search).  On the y grid (t = 0, every coarse candidate) the
// quadratic is A0 itself: the Horner step would add exact zeros, so it is
// skipped with the same result.
// With a lattice of at most 2^24 points per cell (shift <= 24) the cell
// fraction t is one exact float, and the products by t take the float form
// of the double-float product (the same roundings, as t has no low part).
__device__ __forceinline__ Eval eval_table(const Geom& g, const FastView& f,
                                           int64_t i, int64_t nu) {
    const int64_t cell = nu >> g.shift;
    const int64_t p = cell - f.c_lo;
    if ((uint64_t)p >= (uint64_t)(f.n_pos - 1)) return eval_outside(g, f, i, nu);
    const int64_t frac = nu & (g.one - 1);
    const dfloat a0 = f.C0[p];
    const float b = f.Cb[p];
    dfloat S = a0;
    if (frac != 0) {
        if (g.shift <= 24) {
            const float t = __fmul_rn(__int2float_rn((int)frac), f.inv_one_f);   // exact
            S = df_add(a0, df_mul_f(df_add(f.C1[p], df_mul_f(f.C2[p], t)), t));
        } else {
            const dfloat t = df_mul_f(df_from_i64(frac), f.inv_one_f);
            S = df_add(a0, df_mul(t, df_add(f.C1[p], df_mul(t, f.C2[p]))));
        }
    }
    const dfloat a = df_mul(df_from_i64(nu - (i - g.hx) * g.one), dfloat{f.step_hi, f.step_lo});
    const dfloat ctl = df_mul(dfloat{f.kk_hi, f.kk_lo}, df_mul(a, a));
    const dfloat gv = df_add(ctl, S);
    const float beta = b + 3.0e-13f * fabsf(ctl.hi) +
                       f.beta_ctl * (f.k_f * fabsf(a.hi) * 1.0001f) + 4.0e-16f * fabsf(gv.hi);
    return {gv, beta};
}

// The same cost with the cell coefficients formed from the tables (J, which
// runs beside the pass that stores them); the same arithmetic, hence the
// same value.
__device__ __forceinline__ Eval eval_table_direct(const Geom& g, const FastView& f,
                                                  int64_t i, int64_t nu) {
    const int64_t cell = nu >> g.shift;
    const int64_t p = cell - f.c_lo;
    if (p < 0 || p + 1 >= f.n_pos) return eval_outside(g, f, i, nu);
    const dfloat t = df_mul_f(df_from_i64(nu - cell * g.one), f.inv_one_f);
    return eval_poly(g, f, i, nu, t, coef_of(f, p, w2_of(f)));
}

// lanes of this thread's group of G (groups may diverge from each other)
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if (G == 32) return 0xffffffffu;
    return (0xffffffffu >> (32 - G)) << ((threadIdx.x & 31) & ~(G - 1));
}

template <int G>
__device__ __forceinline__ dfloat gmin_df(dfloat v) {
    const unsigned gm = group_mask<G>();
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        dfloat o{__shfl_xor_sync(gm, v.hi, off, G),
                 __shfl_xor_sync(gm, v.lo, off, G)};
        if (df_lt(o, v)) v = o;
    }
    return v;
}
template <int G>
__device__ __forceinline__ int64_t gmin_i64(int64_t v) {
    const unsigned gm = group_mask<G>();
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const int64_t o = __shfl_xor_sync(gm, v, off, G);
        v = o < v ? o : v;
    }
    return v;
}
template <int G>
__device__ __forceinline__ int64_t gmax_i64(int64_t v) {
    const unsigned gm = group_mask<G>();
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const int64_t o = __shfl_xor_sync(gm, v, off, G);
        v = o > v ? o : v;
    }
    return v;
}
template <int G>
__device__ __forceinline__ int32_t gmin_i32(int32_t v) {
    const unsigned gm = group_mask<G>();
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
        v = min(v, __shfl_xor_sync(gm, v, off, G));
    return v;
}
__device__ __forceinline__ bool before(double ga, int32_t pa, double gb,
                                       int32_t pb) {
    return ga < gb || (ga == gb && pa < pb);
}
template <int G>
__device__ __forceinline__ void glex(double& gv, int32_t& pos, int64_t& nu) {
    const unsigned gm = group_mask<G>();
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const double go = __shfl_xor_sync(gm, gv, off, G);
        const int32_t po = __shfl_xor_sync(gm, pos, off, G);
        const int64_t no = __shfl_xor_sync(gm, nu, off, G);
        if (before(go, po, gv, pos)) { gv = go; pos = po; nu = no; }
    }
}

// The running winner: cost interval [gv - beta, gv + beta] (beta 0: exact).
struct Best {
    dfloat gv;
    float beta;
    int32_t pos;
    int64_t nu;
    bool is_exact;  // `exact` holds the serial FP64 cost
    double exact;
};

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

__device__ __forceinline__ dfloat df_pm(dfloat v, float b) { return df_add_f(v, b); }

// All candidates in play re-costed by the serial FP64 quadrature (used when
// more distinct values are in play than the group has lanes).
template <int G, typename CandFn>
__device__ Best resolve_serial(const Geom& g, const FastView& f, int64_t i, int lane,
                               const Best& best, bool have_best, dfloat hi, int p0,
                               int p_end, CandFn cand, int32_t* n_exact,
                               CoopSmem* cs) {
    double xg = DBL_MAX;
    int32_t xp = INT_MAX;
    int64_t xn = 0;
    int M = 0;
    int64_t mnu = 0;
    int32_t mpos = INT_MAX;
    auto flush = [&]() {
        if (M == 0) return;
        const double v = exact_costs_coop<G>(g, f, i, lane, mnu, M, cs);
        if (lane < M && before(v, mpos, xg, xp)) { xg = v; xp = mpos; xn = mnu; }
        if (lane == 0 && n_exact) atomicAdd(n_exact, M);
        M = 0;
    };
    if (have_best && !df_lt(hi, df_pm(best.gv, -best.beta))) {
        if (best.is_exact) {
            if (lane == 0) { xg = best.exact; xp = best.pos; xn = best.nu; }
        } else {
            if (lane == 0) { mnu = best.nu; mpos = best.pos; }
            M = 1;
        }
    }
    const unsigned gm = group_mask<G>();
    const int base = (threadIdx.x & 31) & ~(G - 1);
    for (int pb = p0; pb < p_end; pb += G) {
        const int p = pb + lane;
        bool member = false;
        int64_t nu = 0;
        if (p < p_end) {
            nu = cand(p);
            const Eval e = eval_table(g, f, i, nu);
            member = !df_lt(hi, df_pm(e.gv, -e.beta));
        }
        unsigned mask = (__ballot_sync(gm, member) >> base) & (0xffffffffu >> (32 - G));
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const int64_t cn = __shfl_sync(gm, nu, src, G);
            if (lane == M) { mnu = cn; mpos = pb + src; }
            ++M;
            if (M == kTieBatch) flush();
        }
    }
    flush();
    glex<G>(xg, xp, xn);
    return {df_from_double(xg), 4.0e-15f * (float)fabs(xg), xp, xn, true, xg};
}

// Resolve one stage of the list: the carried winner (lane 0) plus positions
// p0 + lane + k G < p_end.  Returns the first minimum of the serial FP64
// costs over all of them.
constexpr int kKeep = 12;   // candidates per lane whose screened costs are kept
// doubles of shared scratch per lane: kept costs (double-float) and bounds
// (float), or exact-tier terms
constexpr int kGroupScratch = kKeep * 3 / 2 > kTieBatch ? kKeep * 3 / 2 : kTieBatch;
// lanes per x0 point: the screening search, and the deferred (block-
// cooperative) search, whose second tier takes up to kCoopG members at once
constexpr int kFastG = kSearchLanesDefault;
constexpr int kCoopG = 16;

// How resolve() settles a stage with several values still in play:
// kTierDefer gives up (the x0 point is searched again by the deferred
// kernel); kTierCoop runs the second and third tiers with the whole block,
// whose groups all search the same x0 point.
enum TierMode { kTierDefer = 1, kTierCoop = 2 };
constexpr int32_t kDeferPos = -2;   // Best.pos of a deferred search

// A deferred search: the x0 point, the stage whose near-tie stopped it and
// the winner carried into that stage.
struct DeferRec {
    int64_t i;
    int32_t stage;
    Best best;
};
static_assert(sizeof(DeferRec) <= kDeferRecBytes, "deferred-search record size");
constexpr int kSearchT = 128;   // threads per block of the search

template <int G, int Mode, typename CandFn>
__device__ Best resolve(const Geom& g, const FastView& f, int64_t i, int lane,
                        const Best& best, int p0, int p_end, CandFn cand,
                        int32_t* n_exact, double* tie_terms, CoopSmem* cs) {
    const bool have_best = best.pos != INT_MAX;
    // 1. smallest upper end; the costs and bounds of this lane's first kKeep
    // candidates are kept (the rest are evaluated again below), in this
    // lane's column of the group's shared scratch (free until the third
    // tier, which runs after the last use)
    dfloat hi = {FLT_MAX, 0.f};
    if (lane == 0 && have_best) hi = df_pm(best.gv, best.beta);
    dfloat* gv_k = (dfloat*)tie_terms;                 // gv_k[k * G + lane]
    float* be_k = (float*)(gv_k + kKeep * G);          // be_k[k * G + lane]
    // kept rows holding a candidate of this stage (the same for the group)
    const int nk = p_end > p0 ? min(kKeep, (p_end - p0 + G - 1) / G) : 0;
#pragma unroll 2
    for (int k = 0; k < nk; ++k) {
        const int p = p0 + lane + k * G;
        if (p < p_end) {
            const Eval e = eval_table(g, f, i, cand(p));
            const dfloat h = df_pm(e.gv, e.beta);
            if (df_lt(h, hi)) hi = h;
            gv_k[k * G + lane] = e.gv;
            be_k[k * G + lane] = e.beta;
        }
    }
    for (int p = p0 + lane + kKeep * G; p < p_end; p += G) {
        const Eval e = eval_table(g, f, i, cand(p));
        const dfloat h = df_pm(e.gv, e.beta);
        if (df_lt(h, hi)) hi = h;
    }
    hi = gmin_df<G>(hi);
    // 2. distinct values still in play, and their first position
    int64_t vmin = INT64_MAX, vmax = INT64_MIN;
    int32_t pmin = INT_MAX;
    if (lane == 0 && have_best && !df_lt(hi, df_pm(best.gv, -best.beta))) {
        vmin = vmax = best.nu;
        pmin = best.pos;
    }
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        const int p = p0 + lane + k * G;
        if (p < p_end && !df_lt(hi, df_pm(gv_k[k * G + lane], -be_k[k * G + lane]))) {
            const int64_t nu = cand(p);
            vmin = nu < vmin ? nu : vmin;
            vmax = nu > vmax ? nu : vmax;
            pmin = p < pmin ? p : pmin;
        }
    }
    for (int p = p0 + lane + kKeep * G; p < p_end; p += G) {
        const int64_t nu = cand(p);
        const Eval e = eval_table(g, f, i, nu);
        if (!df_lt(hi, df_pm(e.gv, -e.beta))) {
            vmin = nu < vmin ? nu : vmin;
            vmax = nu > vmax ? nu : vmax;
            pmin = p < pmin ? p : pmin;
        }
    }
    // one value in play iff every lane's values in play equal the value at
    // the first position in play (a vote instead of group minima and maxima)
    pmin = gmin_i32<G>(pmin);
    bool one = false;
    int64_t v0 = 0;
    if (pmin != INT_MAX) {
        v0 = (have_best && pmin == best.pos) ? best.nu : cand(pmin);
        one = __all_sync(group_mask<G>(), vmin == INT64_MAX || (vmin == v0 && vmax == v0));
    }
    if (one) {
        // one value in play: its first occurrence wins, with the cost its
        // lane kept (every candidate of that value has the same cost)
        if (have_best && pmin == best.pos) return best;
        const int kk = (pmin - p0) / G, owner = (pmin - p0) % G;
        if (kk < kKeep) {
            __syncwarp(group_mask<G>());
            return {gv_k[kk * G + owner], be_k[kk * G + owner], pmin, v0, false, 0.0};
        }
        const Eval e = eval_table(g, f, i, v0);
        return {e.gv, e.beta, pmin, v0, false, 0.0};
    }
    if (Mode == kTierDefer) return {{0.f, 0.f}, 0.f, kDeferPos, 0, false, 0.0};
    // 3. several values in play.  Gather them into lanes (member m in lane
    // m; the carried winner first), cost each by the direct double-float
    // quadrature (second tier) and keep those whose tighter intervals can
    // still hold the first minimum; if they are one value, its first position
    // wins, otherwise their serial FP64 costs decide (third tier).
    const unsigned gm = group_mask<G>();
    const int base = (threadIdx.x & 31) & ~(G - 1);
    int M = 0;
    bool overflow = false;
    int64_t mnu = 0;
    int32_t mpos = INT_MAX;
    bool mexact = false;
    double mval = 0.0;
    if (have_best && !df_lt(hi, df_pm(best.gv, -best.beta))) {
        if (lane == 0) { mnu = best.nu; mpos = best.pos; mexact = best.is_exact; mval = best.exact; }
        M = 1;
    }
    auto gather = [&](int pb, bool member, int64_t nu) {
        unsigned mask = (__ballot_sync(gm, member) >> base) & (0xffffffffu >> (32 - G));
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const int64_t cn = __shfl_sync(gm, nu, src, G);
            if (M < G) {
                if (lane == M) { mnu = cn; mpos = pb + src; mexact = false; }
                ++M;
            } else {
                overflow = true;
            }
        }
    };
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        const int pb = p0 + k * G;
        {
            const int p = pb + lane;
            const bool member = p < p_end &&
                                !df_lt(hi, df_pm(gv_k[k * G + lane], -be_k[k * G + lane]));
            gather(pb, member, member ? cand(p) : 0);
        }
    }
    for (int pb = p0 + kKeep * G; pb < p_end; pb += G) {
        const int p = pb + lane;
        bool member = false;
        int64_t nu = 0;
        if (p < p_end) {
            nu = cand(p);
            const Eval e = eval_table(g, f, i, nu);
            member = !df_lt(hi, df_pm(e.gv, -e.beta));
        }
        gather(pb, member, nu);
    }
    if (overflow)   // more distinct candidates in play than lanes (rare)
        return resolve_serial<G>(g, f, i, lane, best, have_best, hi, p0, p_end, cand,
                                 n_exact, cs);
    // before the second tier (block-cooperative search): r = the member with
    // the least table cost; when every other member lies in r's cell and is
    // certified above it (diff_df_coop), r wins without the second tier
    int64_t tried = INT64_MIN;   // the r whose certification failed
    if (Mode == kTierCoop) {
        const bool mine = lane < M;
        double rg = DBL_MAX;
        float rb = 0.f;
        if (mine) {
            const Eval e = eval_table(g, f, i, mnu);
            rg = mexact ? mval : df_to_double(e.gv);
            rb = mexact ? 0.f : e.beta;
        }
        int32_t rp = mine ? mpos : INT_MAX;
        int64_t rn = mine ? mnu : 0;
        glex<G>(rg, rp, rn);
        const int64_t rcell = rn >> g.shift, rpp = rcell - f.c_lo;
        const bool other = mine && mnu != rn;
        const bool far = other && (mnu >> g.shift) != rcell;
        bool cert = rpp >= 0 && rpp + 1 < f.n_pos && !__any_sync(gm, far);
        unsigned om = (__ballot_sync(gm, other) >> base) & (0xffffffffu >> (32 - G));
        const bool attempted = cert && om;
        while (cert && om) {
            const int src = __ffs(om) - 1;
            om &= om - 1;
            double dlt, thr;
            diff_df_coop<G>(g, f, i, rn, __shfl_sync(gm, mnu, src, G), lane, cs, dlt, thr);
            cert = dlt > thr;
        }
        if (cert) {
            const unsigned wmask = (__ballot_sync(gm, mine && mpos == rp) >> base) &
                                   (0xffffffffu >> (32 - G));
            const float wb = __shfl_sync(gm, rb, __ffs(wmask) - 1, G);
            return {df_from_double(rg), wb, rp, rn, false, 0.0};
        }
        if (attempted) tried = rn;
    }
    // second tier
    double g2 = 0.0, b2 = 0.0;
    if (lane == 0 && n_exact && f.n_tier2) atomicAdd(f.n_tier2, M);
    for (int m = 0; m < M; m += 2) {
        const int m1 = m + 1 < M ? m + 1 : m;
        const int64_t cn[2] = {__shfl_sync(gm, mnu, m, G), __shfl_sync(gm, mnu, m1, G)};
        double v[2], bv[2];
        direct_df_cost2<G>(g, f, i, cn, lane, v, bv, Mode == kTierCoop ? cs : nullptr);
        if (lane == m) { g2 = v[0]; b2 = bv[0]; }
        if (m1 != m && lane == m1) { g2 = v[1]; b2 = bv[1]; }
    }
    if (lane < M && mexact) { g2 = mval; b2 = 0.0; }   // serial cost already known
    double hi2 = lane < M ? g2 + b2 : DBL_MAX;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
        hi2 = fmin(hi2, __shfl_xor_sync(gm, hi2, off, G));
    const bool in2 = lane < M && g2 - b2 <= hi2;
    int64_t v2min = in2 ? mnu : INT64_MAX, v2max = in2 ? mnu : INT64_MIN;
    int32_t p2min = in2 ? mpos : INT_MAX;
    v2min = gmin_i64<G>(v2min);
    v2max = gmax_i64<G>(v2max);
    p2min = gmin_i32<G>(p2min);
    if (v2min == v2max) {
        if (have_best && p2min == best.pos) return best;
        const unsigned wmask = (__ballot_sync(gm, in2 && mpos == p2min) >> base) &
                               (0xffffffffu >> (32 - G));
        const int wl = __ffs(wmask) - 1;
        const double wg = __shfl_sync(gm, g2, wl, G);
        const double wb = __shfl_sync(gm, b2, wl, G);
        return {df_from_double(wg), (float)(wb + 4.0e-15 * fabs(wg)) * 1.0001f, p2min,
                v2min, false, 0.0};
    }
    // between the tiers (block-cooperative search): r = the first least
    // second-tier cost in play; when every other member in play lies in r's
    // cell and its cost difference to r is certified positive (diff_df_coop),
    // r is the first minimum of the serial costs and no serial cost is formed
    if (Mode == kTierCoop) {
        const bool mine = lane < M && in2;
        double rg = mine ? g2 : DBL_MAX;
        int32_t rp = mine ? mpos : INT_MAX;
        int64_t rn = mine ? mnu : 0;
        glex<G>(rg, rp, rn);
        const int64_t rcell = rn >> g.shift, rpp = rcell - f.c_lo;
        const bool other = mine && mnu != rn;
        const bool far = other && (mnu >> g.shift) != rcell;
        bool cert = rn != tried && rpp >= 0 && rpp + 1 < f.n_pos && !__any_sync(gm, far);
        unsigned om = (__ballot_sync(gm, other) >> base) & (0xffffffffu >> (32 - G));
        while (cert && om) {
            const int src = __ffs(om) - 1;
            om &= om - 1;
            double dlt, thr;
            diff_df_coop<G>(g, f, i, rn, __shfl_sync(gm, mnu, src, G), lane, cs, dlt, thr);
            cert = dlt > thr;
        }
        if (cert) {
            const unsigned wmask = (__ballot_sync(gm, mine && mpos == rp) >> base) &
                                   (0xffffffffu >> (32 - G));
            const int wl = __ffs(wmask) - 1;
            const double wb = __shfl_sync(gm, b2, wl, G);
            return {df_from_double(rg), (float)(wb + 4.0e-15 * fabs(rg)) * 1.0001f, rp, rn,
                    false, 0.0};
        }
    }
    // third tier: serial FP64 costs of the members still in play
    double xg = DBL_MAX;
    int32_t xp = INT_MAX;
    int64_t xn = 0;
    if (lane < M && in2 && mexact) { xg = mval; xp = mpos; xn = mnu; }
    const bool need = in2 && !mexact;
    const unsigned nmask = (__ballot_sync(gm, need) >> base) & (0xffffffffu >> (32 - G));
    int K = 0;
    int64_t knu = 0;
    int32_t kpos = INT_MAX;
    unsigned rest = nmask;
    while (rest) {
        const int src = __ffs(rest) - 1;
        rest &= rest - 1;
        const int64_t cn = __shfl_sync(gm, mnu, src, G);
        const int32_t cp = __shfl_sync(gm, mpos, src, G);
        if (lane == K) { knu = cn; kpos = cp; }
        ++K;
        if (K == kTieBatch || rest == 0) {
            const double v = exact_costs_coop<G>(g, f, i, lane, knu, K, cs);
            if (lane < K && before(v, kpos, xg, xp)) { xg = v; xp = kpos; xn = knu; }
            if (lane == 0 && n_exact) atomicAdd(n_exact, K);
            K = 0;
        }
    }
    glex<G>(xg, xp, xn);
    return {df_from_double(xg), 4.0e-15f * (float)fabs(xg), xp, xn, true, xg};
}

// Corollary 1's pointwise argmin for x0 point i over eq. (2)'s list: stage 0
// (previous value, neighbours, coarse set), then the refinement levels
// around the running winner, from stage `stage0` with carried winner `best`.
// The group's lane 0 of a `writer` group stores the result; a deferred
// search records where it stopped instead.
template <int G, int Mode>
__device__ __forceinline__ void search_one(const Geom& g, const FastView& f,
                                           const int64_t* __restrict__ nu_pre,
                                           int64_t* __restrict__ nu_out,
                                           int32_t* __restrict__ idx_out,
                                           int32_t* n_exact, double* tie_terms,
                                           CoopSmem* cs, int64_t i, bool active,
                                           bool writer, int stage0, Best best) {
    const int lane = threadIdx.x & (G - 1);
    const int64_t ic = active ? i : g.n_x - 1;
    const int64_t* coarse = f.coarse;
    int32_t* cnt = active && writer ? n_exact : nullptr;
    const int n0 = 1 + 2 * g.n_nbr + g.n_coarse;
    const int R = g.n_refine;   // candidates per refinement level
    const int half = R / 2;
    Best carried = best;
    int stage = stage0;
    for (; stage <= g.n_levels; ++stage) {
        carried = best;
        if (stage == 0) {
            best = resolve<G, Mode>(g, f, ic, lane, best, 0, n0,
                                    [&](int p) { return stage0_nu(g, nu_pre, coarse, ic, p); },
                                    cnt, tie_terms, cs);
        } else {
            const int64_t h = g.q << (g.bits * (g.n_levels - stage));
            const int64_t centre = best.nu;
            const int pos = n0 + (stage - 1) * R;
            best = resolve<G, Mode>(g, f, ic, lane, best, pos, pos + R,
                                    [&](int p) {
                                        const int k = p - pos;
                                        const int64_t m = k < half ? k - half : k - half + 1;
                                        return centre + m * h;
                                    },
                                    cnt, tie_terms, cs);
        }
        if (best.pos == kDeferPos) break;
    }
    if (!active || !writer || lane != 0) return;
    if (best.pos == kDeferPos) {
        DeferRec* rec = (DeferRec*)f.defer_list;
        rec[atomicAdd(f.defer_cnt, 1)] = {i, stage, carried};
        return;
    }
    nu_out[i] = best.nu;
    idx_out[i] = best.pos;
}

// One group of G lanes per x0 point; near-ties are deferred.
// Points i_lo .. i_hi - 1 (i_hi < 0: every point) are searched.
template <int G>
__device__ __forceinline__ void search_body(const Geom& g, const FastView& f,
                                            const int64_t* __restrict__ nu_pre,
                                            int64_t* __restrict__ nu_out,
                                            int32_t* __restrict__ idx_out,
                                            int32_t* n_exact, double* tie_smem,
                                            int64_t bx, int64_t i_lo = 0, int64_t i_hi = -1) {
    const int64_t i = i_lo + (bx * blockDim.x + threadIdx.x) / G;
    const int64_t hi = i_hi < 0 ? g.n_x : i_hi;
    double* tie_terms = tie_smem + (threadIdx.x / G) * (kGroupScratch * G);
    const Best none{{FLT_MAX, 0.f}, 0.f, INT_MAX, 0, false, 0.0};
    search_one<G, kTierDefer>(g, f, nu_pre, nu_out, idx_out, n_exact, tie_terms,
                              nullptr, i, i < hi, true, 0, none);
}

// The deferred x0 points, one per block at a time (blocks bx, bx + nbx, ...
// of the list), each resumed at the stage that stopped it: every group of
// the block searches the same point, the second tier is split over the
// block, group 0 stores the result.
template <int G>
__device__ __forceinline__ void search_deferred_body(const Geom& g, const FastView& f,
                                                     const int64_t* __restrict__ nu_pre,
                                                     int64_t* __restrict__ nu_out,
                                                     int32_t* __restrict__ idx_out,
                                                     int32_t* n_exact, double* tie_smem,
                                                     CoopSmem& cs, int64_t bx,
                                                     int64_t nbx) {
    const int n = *(volatile int32_t*)f.defer_cnt;
    double* tie_terms = tie_smem + (threadIdx.x / G) * (kGroupScratch * G);
    const DeferRec* rec = (const DeferRec*)f.defer_list;
    for (int64_t k = bx; k < n; k += nbx) {
        const DeferRec r = rec[k];
        search_one<G, kTierCoop>(g, f, nu_pre, nu_out, idx_out, n_exact, tie_terms,
                                 &cs, r.i, true, threadIdx.x < G, r.stage, r.best);
        __syncthreads();   // tie_smem and cs are reused by the next point
    }
}

template <int G>
__global__ void __launch_bounds__(kSearchT, 6) k_search_fast(Geom g, FastView f,
                                                     const int64_t* __restrict__ nu_pre,
                                                     int64_t* __restrict__ nu_out,
                                                     int32_t* __restrict__ idx_out,
                                                     int32_t* n_exact, int64_t i_lo,
                                                     int64_t i_hi) {
    __shared__ double tie_smem[kSearchT * kGroupScratch];
    search_body<G>(g, f, nu_pre, nu_out, idx_out, n_exact, tie_smem, blockIdx.x, i_lo,
                   i_hi);
}

// Blocks of the deferred search of one instance: one per 128 x0 points
// (fine grids defer many points at their last levels), at least 64, at most
// four per SM.
static unsigned defer_blocks_of(const Geom& g) {
    const int64_t b = g.n_x / 128;
    return (unsigned)std::max<int64_t>(64, std::min<int64_t>(b, 4 * (int64_t)sm_count()));
}

__global__ void __launch_bounds__(kCoopT, 2) k_search_deferred(Geom g, FastView f,
                                                           const int64_t* __restrict__ nu_pre,
                                                           int64_t* __restrict__ nu_out,
                                                           int32_t* __restrict__ idx_out,
                                                           int32_t* n_exact) {
    __shared__ double tie_smem[kCoopT * kGroupScratch];
    __shared__ CoopSmem cs;
    if (threadIdx.x == 0) cs.scratch = tie_smem;
    __syncthreads();
    search_deferred_body<kCoopG>(g, f, nu_pre, nu_out, idx_out, n_exact, tie_smem, cs,
                                 blockIdx.x, gridDim.x);
}

// Per-instance constants: a_l = phi_l w_l and phi_l in double-float, the
// prior exponent x_i^2 / 2 sigma^2 and the constant table (df_exp's
// exp(k/64), the inverse factorials).  W2 = sum phi_l w_l^2 is formed with
// the filter slices (kernels_tc.cu).
static_assert(kConstTab <= 128, "constant table within the set-up blocks");
__device__ __forceinline__ void fast_setup_elem(const Geom& g, const FastView& f, int64_t k) {
    if (k < g.n_w) {
        const double w = (double)(k - g.hw) * g.delta;
        f.a[k] = df_from_double(f.phi[k] * w);
        f.phidf[k] = df_from_double(f.phi[k]);
        f.wdf[k] = df_from_double(w);
    }
    if (k < g.n_x) {
        const double x = x_of(g, k);
        f.prior[k] = df_from_double(__ddiv_rn(__dmul_rn(x, x), g.two_s2));
    }
    if (k < kConstTab) f.t64[k] = const_table_entry((int)k);
}

__global__ void k_fast_setup(Geom g, FastView f) {
    fast_setup_elem(g, f, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(256) kb_fast_setup(const SetupDev* descs,
                                                     const BlockRef* map) {
    const BlockRef r = map[blockIdx.x];
    const SetupDev& d = descs[r.inst];
    fast_setup_elem(d.g, d.f, (int64_t)r.local * blockDim.x + threadIdx.x);
}

// ---- J --------------------------------------------------------------------

constexpr int kJThreads = 256;
// J = sum_i p_i g(f_i; x_i): block partials (fixed tree), then the last
// block to finish adds the partials (lane-strided, then a warp tree).  Returns true in thread
// 0 of that block, with J in *J_out (the counter is left at zero).
__device__ __forceinline__ bool J_partial_body(const Geom& g, const FastView& f,
                                               const double* __restrict__ px,
                                               const int64_t* __restrict__ nu,
                                               double* red, int* last, int64_t bx,
                                               double* J_out) {
    const int64_t i = bx * kJThreads + threadIdx.x;
    double v = 0.0;
    if (i < g.n_x) v = px[i] * df_to_double(eval_table_direct(g, f, i, nu[i]).gv);
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = kJThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        f.Jpart[bx] = red[0];
        __threadfence();
        *last = atomicAdd(f.J_done, 1) == (int)(f.J_blocks - 1);
    }
    __syncthreads();
    if (!*last || threadIdx.x >= 32) return false;
    __threadfence();
    // the block partials: lane-strided sums, then a warp tree (fixed order)
    double sum = 0.0;
    for (int64_t b = threadIdx.x; b < f.J_blocks; b += 32) sum += __ldcg(f.Jpart + b);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off);
    if (threadIdx.x != 0) return false;
    *J_out = sum;
    *f.J_done = 0;
    return true;
}

// Cell coefficients of the new tables for the next search (blocks after the
// J blocks of the same launch).
__device__ __forceinline__ void cells_body(const FastView& f, int64_t bx) {
    const int64_t p = bx * kJThreads + threadIdx.x;
    if (p + 1 >= f.n_pos) return;
    const Coef c = coef_of(f, p, w2_of(f));
    f.C0[p] = c.a0;
    f.C1[p] = c.a1;
    f.C2[p] = c.a2;
    f.Cb[p] = c.b;
}

// J into *out; also empties the deferred-search list for the next sweep.
// Blocks from J_blocks on store the cell coefficients.
__global__ void __launch_bounds__(kJThreads) k_J_partial(Geom g, FastView f,
                                                         const double* __restrict__ px,
                                                         const int64_t* __restrict__ nu,
                                                         double* out) {
    __shared__ double red[kJThreads];
    __shared__ int last;
    if (blockIdx.x >= f.J_blocks) {
        cells_body(f, blockIdx.x - f.J_blocks);
        return;
    }
    double J;
    if (J_partial_body(g, f, px, nu, red, &last, blockIdx.x, &J)) {
        *out = J;
        *f.defer_cnt = 0;
    }
}


// ---- batched wrappers -------------------------------------------------------
// Every block of a batched launch works on one instance: the block map gives
// (instance, block of that instance's own grid); the instance descriptor is
// staged in shared memory and the single-instance body runs unchanged.

__device__ __forceinline__ BlockRef stage(const InstDev* insts, const BlockRef* map,
                                          InstDev& sd) {
    const BlockRef r = map[blockIdx.x];
    const int* src = (const int*)(insts + r.inst);
    int* dst = (int*)&sd;
    for (int k = threadIdx.x; k < (int)(sizeof(InstDev) / 4); k += blockDim.x)
        dst[k] = src[k];
    __syncthreads();
    return r;
}

template <int G>
__global__ void __launch_bounds__(kSearchT, 6) kb_search(const InstDev* insts, const BlockRef* map) {
    __shared__ InstDev sd;
    const BlockRef r = stage(insts, map, sd);
    __shared__ double tie_smem[kSearchT * kGroupScratch];
    search_body<G>(sd.g, sd.f, sd.nu[sd.cur], sd.nu[sd.cur ^ 1], sd.idx, sd.f.n_exact,
                   tie_smem, r.local);
}

__global__ void __launch_bounds__(kCoopT, 2) kb_search_deferred(const InstDev* insts,
                                                            const BlockRef* map) {
    __shared__ InstDev sd;
    const BlockRef r = stage(insts, map, sd);
    __shared__ double tie_smem[kCoopT * kGroupScratch];
    __shared__ CoopSmem cs;
    if (threadIdx.x == 0) cs.scratch = tie_smem;
    __syncthreads();
    search_deferred_body<kCoopG>(sd.g, sd.f, sd.nu[sd.cur], sd.nu[sd.cur ^ 1], sd.idx,
                                 sd.f.n_exact, tie_smem, cs, r.local, sd.defer_blocks);
}

// Last kernel of a batched sweep: J into its history slot, then the sweep
// counter and the double buffer advance (by the instance's last J block).
__global__ void __launch_bounds__(kJThreads) kb_J_partial(InstDev* insts,
                                                          const BlockRef* map) {
    __shared__ InstDev sd;
    __shared__ double red[kJThreads];
    __shared__ int last;
    const BlockRef r = stage(insts, map, sd);
    if (r.local >= sd.f.J_blocks) {
        cells_body(sd.f, r.local - sd.f.J_blocks);
        return;
    }
    double J;
    if (J_partial_body(sd.g, sd.f, sd.px, sd.nu[sd.cur ^ 1], red, &last, r.local, &J)) {
        InstDev& d = insts[r.inst];
        d.J[d.sweeps + 1] = J;
        d.sweeps += 1;
        d.cur ^= 1;
        *d.f.defer_cnt = 0;
    }
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
    u1_plan(g, 32, fp);
    fp->J_blocks = (g.n_x + kJThreads - 1) / kJThreads;
    fp->cell_blocks = (fp->n_pos - 1 + kJThreads - 1) / kJThreads;
    tc_plan(g, fp);
}

void launch_fast_setup(const Geom& g, const FastView& f, cudaStream_t s) {
    int64_t n = g.n_w > g.n_x ? g.n_w : g.n_x;
    n = n > kConstTab ? n : kConstTab;
    k_fast_setup<<<blocks(n, 256), 256, 0, s>>>(g, f);
}

void launch_batch_setup_fast(const SetupLaunch& sl, cudaStream_t s) {
    if (sl.elem_blocks)
        kb_fast_setup<<<(unsigned)sl.elem_blocks, 256, 0, s>>>(sl.descs, sl.elem_map);
}

void launch_search_fast(const Geom& g, const FastView& f, const int64_t* nu_in,
                        int64_t* nu_out, int32_t* idx, cudaStream_t s, int64_t i_lo,
                        int64_t i_hi, const LaunchCfg* cfg) {
    const int64_t hi = i_hi < 0 ? g.n_x : i_hi;
    const int G = cfg && cfg->search_lanes ? cfg->search_lanes : kFastG;
    const int64_t threads = (hi - i_lo) * (int64_t)G;
    if (threads <= 0) return;
    const unsigned nb = blocks(threads, kSearchT);
    switch (G) {
        case 4: k_search_fast<4><<<nb, kSearchT, 0, s>>>(g, f, nu_in, nu_out, idx, f.n_exact,
                                                        i_lo, hi); break;
        case 16: k_search_fast<16><<<nb, kSearchT, 0, s>>>(g, f, nu_in, nu_out, idx,
                                                          f.n_exact, i_lo, hi); break;
        default: k_search_fast<8><<<nb, kSearchT, 0, s>>>(g, f, nu_in, nu_out, idx, f.n_exact,
                                                         i_lo, hi); break;
    }
    const unsigned nd = cfg && cfg->defer_blocks ? (unsigned)cfg->defer_blocks
                                                 : defer_blocks_of(g);
    k_search_deferred<<<nd, kCoopT, 0, s>>>(g, f, nu_in, nu_out, idx, f.n_exact);
}

int64_t search_blocks(const Geom& g, int lanes) {
    return (g.n_x * lanes + kSearchT - 1) / kSearchT;
}

int64_t batch_blocks(const Geom& g, const FastPlan& fp, int kind) {
    switch (kind) {
        case kBSearch: return search_blocks(g, kFastG);
        case kBTile:
        case kBRun: return u1_batch_blocks(g, fp, kind);
        case kBPerY: return (g.n_y + 255) / 256;
        case kBTabPart: return tc_table_blocks(fp);
        case kBTabComb: return tc_combine_blocks(fp);
        case kBBuildE: return tc_build_E_blocks(g, fp);
        case kBJPart: return fp.J_blocks + fp.cell_blocks;
    }
    return 0;
}

void launch_batch_sweep(const BatchLaunch& bl, cudaStream_t s, Prof* prof) {
    launch_batch_search(bl, s, prof);
    launch_batch_rest(bl, s, prof);
}

void launch_batch_search(const BatchLaunch& bl, cudaStream_t s, Prof* prof) {
    const InstDev* d = bl.insts;
    ProfScope ps(prof, "search");
    if (bl.search_blocks) {
        const unsigned nb = (unsigned)bl.search_blocks;
        switch (bl.search_lanes) {
            case 4: kb_search<4><<<nb, kSearchT, 0, s>>>(d, bl.search_map); break;
            case 16: kb_search<16><<<nb, kSearchT, 0, s>>>(d, bl.search_map); break;
            default: kb_search<8><<<nb, kSearchT, 0, s>>>(d, bl.search_map); break;
        }
    }
    if (bl.defer_blocks)
        kb_search_deferred<<<(unsigned)bl.defer_blocks, kCoopT, 0, s>>>(d, bl.defer_map);
}

void launch_batch_rest(const BatchLaunch& bl, cudaStream_t s, Prof* prof) {
    launch_batch_u1(bl, s, prof);
    launch_batch_tables(bl, s, prof);
    ProfScope ps(prof, "J");
    kb_J_partial<<<(unsigned)bl.n_blocks[kBJPart], kJThreads, 0, s>>>(bl.insts,
                                                                   bl.map[kBJPart]);
}

void launch_J_fast(const Geom& g, const FastView& f, const double* px,
                   const int64_t* nu, double* out, cudaStream_t s, Prof* prof) {
    cudaEvent_t ev;
    int k = prof ? prof->begin("J", &ev) : -1;
    k_J_partial<<<(unsigned)(f.J_blocks + f.cell_blocks), kJThreads, 0, s>>>(g, f, px, nu, out);
    if (prof) prof->end(k, ev);
}

}  // namespace ucp
