// kernels_2d.cu -- the sweep on the 2-dimensional Witsenhausen counterexample
// (Section V-D): x, u and y in R^2, x1 = x0 + u0(x0), y1 = x1 + w,
// x2 = x1 - u1(y1), J = (1/2) E[k^2 |u0|^2 + |x2|^2], x0 ~ N(0, sigma^2 I),
// w ~ N(0, I).  FP64 throughout (the plain path of the one-dimensional
// sweep, in two dimensions), every operation rounded once and every sum in a
// fixed order, so that the decisions are the FP64 ones:
//   - u0 step (Corollary 1, eq. (2), Section IV-A): for every x0 point, the
//     first minimiser of g(u; x) = k^2 |u - x|^2 + S(u), S(u) = sum_cd
//     phi_c phi_d |u - U^(u + w_cd)|^2 with U^ the bilinear interpolant of the
//     u1 table (held constant beyond it), over the list: incumbent; the
//     neighbouring samples of the (2r + 1)^2 window; a coarse 2-D grid; levels
//     of the 3 x 3 window around the best so far at halving steps;
//   - u1 step: U(y) = E[x1 | y1 = y] per component (Section IV-C);
//   - J in index order.
// Layout: x0 point (a, b) has flat index a n_x + b; controllers are int64
// lattice pairs nu[2 i + k] (value nu delta 2^-shift); the u1 table U[2 t + k]
// over flat y indices t; noise weights phi2[c n_w + d] = phi_c phi_d.
#include <float.h>
#include <limits.h>

#include "fixed_sum.cuh"
#include "ucp_2d.h"

namespace ucp {

namespace {

__device__ __forceinline__ double inv_one2(const G2& g) {
    return __longlong_as_double((int64_t)(1023 - g.shift) << 52);  // 2^-shift
}
__device__ __forceinline__ double val2(const G2& g, int64_t nu) {
    return __dmul_rn(__dmul_rn((double)nu, g.delta), inv_one2(g));
}
__device__ __forceinline__ double grid2(const G2& g, int64_t a, int64_t h) {
    return __dmul_rn((double)(a - h), g.delta);
}
__device__ __forceinline__ int64_t clampy(const G2& g, int64_t j) {
    return j < 0 ? 0 : (j > g.n_y - 1 ? g.n_y - 1 : j);
}

// Bilinear interpolation of component k at y-cell (j1, j2) + (t1, t2): along
// axis 2 on both rows, then along axis 1.
__device__ __forceinline__ double bilerp2(const G2& g, const double* __restrict__ U, int k,
                                          int64_t j1, int64_t j2, double t1, double t2) {
    const int64_t n = g.n_y;
    const int64_t a0 = clampy(g, j1), a1 = clampy(g, j1 + 1);
    const int64_t b0 = clampy(g, j2), b1 = clampy(g, j2 + 1);
    const double u00 = U[2 * (a0 * n + b0) + k], u01 = U[2 * (a0 * n + b1) + k];
    const double u10 = U[2 * (a1 * n + b0) + k], u11 = U[2 * (a1 * n + b1) + k];
    const double r0 = __dadd_rn(u00, __dmul_rn(t2, __dsub_rn(u01, u00)));
    const double r1 = __dadd_rn(u10, __dmul_rn(t2, __dsub_rn(u11, u10)));
    return __dadd_rn(r0, __dmul_rn(t1, __dsub_rn(r1, r0)));
}

// S(u) at the lattice pair (nu1, nu2): taps in row-major order, the fixed sum.
__device__ double S2d(const G2& g, const double* __restrict__ phi2,
                      const double* __restrict__ U, int64_t nu1, int64_t nu2) {
    const int64_t c1 = nu1 >> g.shift, c2 = nu2 >> g.shift;   // floor division
    const double t1 = __dmul_rn((double)(nu1 - (c1 << g.shift)), inv_one2(g));
    const double t2 = __dmul_rn((double)(nu2 - (c2 << g.shift)), inv_one2(g));
    const int64_t jb1 = c1 - g.hw + g.hy, jb2 = c2 - g.hw + g.hy;
    const double u1 = val2(g, nu1), u2 = val2(g, nu2);
    const int64_t m = g.n_w;
    FixedSum acc;
    for (int64_t c = 0; c < m; ++c)
        for (int64_t d = 0; d < m; ++d) {
            const double e1 = __dsub_rn(u1, bilerp2(g, U, 0, jb1 + c, jb2 + d, t1, t2));
            const double e2 = __dsub_rn(u2, bilerp2(g, U, 1, jb1 + c, jb2 + d, t1, t2));
            acc.add(__dmul_rn(phi2[c * m + d], __dadd_rn(__dmul_rn(e1, e1), __dmul_rn(e2, e2))));
        }
    return acc.result();
}

__device__ __forceinline__ double cost2d(const G2& g, const double* __restrict__ phi2,
                                         const double* __restrict__ U, int64_t i,
                                         int64_t nu1, int64_t nu2) {
    const double d1 = __dsub_rn(val2(g, nu1), grid2(g, i / g.n_x, g.hx));
    const double d2 = __dsub_rn(val2(g, nu2), grid2(g, i % g.n_x, g.hx));
    return __dadd_rn(__dmul_rn(g.kk, __dadd_rn(__dmul_rn(d1, d1), __dmul_rn(d2, d2))),
                     S2d(g, phi2, U, nu1, nu2));
}

__device__ __forceinline__ bool before2(double ga, int32_t pa, double gb, int32_t pb) {
    return ga < gb || (ga == gb && pa < pb);
}

// Candidate p of stage 0 (incumbent, window, coarse grid) of point i.
__device__ __forceinline__ void stage0_cand(const G2& g, const int64_t* __restrict__ nu_pre,
                                            int64_t i, int p, int64_t& n1, int64_t& n2) {
    const int64_t r = g.n_nbr, side = 2 * r + 1, win = side * side;
    if (p == 0) {
        n1 = nu_pre[2 * i];
        n2 = nu_pre[2 * i + 1];
        return;
    }
    if (p < win) {
        const int64_t k0 = p - 1, centre = r * side + r;
        const int64_t k = k0 < centre ? k0 : k0 + 1;       // the window, centre skipped
        const int64_t a = i / g.n_x + k / side - r, b = i % g.n_x + k % side - r;
        const int64_t j = (a < 0 || a >= g.n_x || b < 0 || b >= g.n_x) ? i : a * g.n_x + b;
        n1 = nu_pre[2 * j];
        n2 = nu_pre[2 * j + 1];
        return;
    }
    const int64_t ci = p - win, nc = g.n_coarse, hq = g.q / 2;
    n1 = (2 * (ci / nc) - (nc - 1)) * hq * g.one;
    n2 = (2 * (ci % nc) - (nc - 1)) * hq * g.one;
}

// One warp per x0 point: the lanes cost the candidates of a stage side by
// side (each candidate's quadrature serial, in the fixed order), the first
// minimum in list order is found by a lexicographic (cost, position) warp
// reduction, then each level's 8 candidates take lanes 0..7.
constexpr int kSearch2T = 128;
__global__ void __launch_bounds__(kSearch2T) k2_search(G2 g, const double* __restrict__ phi2,
                                                       const double* __restrict__ U,
                                                       const int64_t* __restrict__ nu_pre,
                                                       int64_t* __restrict__ nu_out,
                                                       int32_t* __restrict__ idx_out) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (i >= g.n_x * g.n_x) return;   // the same for the warp
    const int64_t side = 2 * (int64_t)g.n_nbr + 1;
    const int n0 = (int)(side * side + (int64_t)g.n_coarse * g.n_coarse);
    double bg = DBL_MAX;
    int32_t bp = INT_MAX;
    int64_t b1 = 0, b2 = 0;
    for (int p = lane; p < n0; p += 32) {
        int64_t n1, n2;
        stage0_cand(g, nu_pre, i, p, n1, n2);
        const double c = cost2d(g, phi2, U, i, n1, n2);
        if (before2(c, p, bg, bp)) { bg = c; bp = p; b1 = n1; b2 = n2; }
    }
    auto reduce = [&]() {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double og = __shfl_xor_sync(0xffffffffu, bg, off);
            const int32_t op = __shfl_xor_sync(0xffffffffu, bp, off);
            const int64_t o1 = __shfl_xor_sync(0xffffffffu, b1, off);
            const int64_t o2 = __shfl_xor_sync(0xffffffffu, b2, off);
            if (before2(og, op, bg, bp)) { bg = og; bp = op; b1 = o1; b2 = o2; }
        }
    };
    reduce();
    int pos = n0;
    for (int lv = 1; lv <= g.n_levels; ++lv) {
        const int64_t h = g.q << (g.n_levels - lv);
        if (lane < 8) {
            const int k9 = lane < 4 ? lane : lane + 1;       // 3 x 3 window, centre skipped
            const int64_t n1 = b1 + (int64_t)(k9 / 3 - 1) * h;
            const int64_t n2 = b2 + (int64_t)(k9 % 3 - 1) * h;
            const double c = cost2d(g, phi2, U, i, n1, n2);
            if (before2(c, pos + lane, bg, bp)) { bg = c; bp = pos + lane; b1 = n1; b2 = n2; }
        }
        reduce();
        pos += 8;
    }
    if (lane == 0) {
        nu_out[2 * i] = b1;
        nu_out[2 * i + 1] = b2;
        idx_out[i] = bp;
    }
}

// u1 step, one thread per target t: the exponents' minimum over the sources,
// then the two numerators and the denominator in source order.
__global__ void __launch_bounds__(128) k2_mmse(G2 g, const int64_t* __restrict__ nu,
                                               double* __restrict__ U) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n_y * g.n_y) return;
    const double two_s2 = __dmul_rn(__dmul_rn(2.0, g.sigma), g.sigma);
    const double y1 = grid2(g, t / g.n_y, g.hy), y2 = grid2(g, t % g.n_y, g.hy);
    const int64_t n = g.n_x * g.n_x;
    auto expo = [&](int64_t i, double& f1, double& f2) {
        const double xa = grid2(g, i / g.n_x, g.hx), xb = grid2(g, i % g.n_x, g.hx);
        f1 = val2(g, nu[2 * i]);
        f2 = val2(g, nu[2 * i + 1]);
        const double d1 = __dsub_rn(y1, f1), d2 = __dsub_rn(y2, f2);
        return __dadd_rn(__ddiv_rn(__dadd_rn(__dmul_rn(xa, xa), __dmul_rn(xb, xb)), two_s2),
                         __ddiv_rn(__dadd_rn(__dmul_rn(d1, d1), __dmul_rn(d2, d2)), 2.0));
    };
    double emin = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double f1, f2;
        const double e = expo(i, f1, f2);
        if (e < emin) emin = e;
    }
    double a1 = 0.0, a2 = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double f1, f2;
        const double w = exp(-__dsub_rn(expo(i, f1, f2), emin));
        a1 = __dadd_rn(a1, __dmul_rn(w, f1));
        a2 = __dadd_rn(a2, __dmul_rn(w, f2));
        den = __dadd_rn(den, w);
    }
    U[2 * t] = __ddiv_rn(a1, den);
    U[2 * t + 1] = __ddiv_rn(a2, den);
}

// The marginal cost at every point's own value (J's terms).
__global__ void __launch_bounds__(128) k2_costs(G2 g, const double* __restrict__ phi2,
                                                const double* __restrict__ U,
                                                const int64_t* __restrict__ nu,
                                                double* __restrict__ terms) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_x * g.n_x) return;
    terms[i] = cost2d(g, phi2, U, i, nu[2 * i], nu[2 * i + 1]);
}

// J = (1/2) sum_i p_i g_i in index order (one thread: the order is the
// definition's).
__global__ void k2_J(G2 g, const double* __restrict__ px, const double* __restrict__ terms,
                     double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int64_t n = g.n_x * g.n_x;
    double J = 0.0;
    for (int64_t i = 0; i < n; ++i) J = __dadd_rn(J, __dmul_rn(px[i], terms[i]));
    *out = __dmul_rn(0.5, J);
}

// ---- set-up -----------------------------------------------------------------

// Exponentials of the prior (i < n_x^2) and of the one-dimensional noise
// weights (the first n_w threads), as the oracle forms them.
__global__ void k2_exps(G2 g, double* __restrict__ pr, double* __restrict__ p1) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.n_x * g.n_x) {
        const double xa = grid2(g, i / g.n_x, g.hx), xb = grid2(g, i % g.n_x, g.hx);
        const double s2 = __dmul_rn(g.sigma, g.sigma);
        pr[i] = exp(__ddiv_rn(-__dadd_rn(__dmul_rn(xa, xa), __dmul_rn(xb, xb)),
                              __dmul_rn(2.0, s2)));
    }
    if (i < g.n_w) {
        const double w = grid2(g, i, g.hw);
        p1[i] = exp(__ddiv_rn(-__dmul_rn(w, w), 2.0));
    }
}

// out = sum of v[0..n) in the fixed order (32-term chunks left to right, then
// pairwise by levels): one block, chunk sums in shared memory, each level's
// additions spread over the block.
__global__ void k2_fixed_sum(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
    extern __shared__ double ch[];
    const int64_t m = sum_chunks(n);
    for (int64_t k = threadIdx.x; k < m; k += blockDim.x) {
        double a = 0.0;
        const int64_t e = min((k + 1) * kSumChunk, n);
        for (int64_t j = k * kSumChunk; j < e; ++j) a = __dadd_rn(a, v[j]);
        ch[k] = a;
    }
    __syncthreads();
    for (int64_t w = m; w > 1;) {
        const int64_t h = w / 2;
        for (int64_t k0 = 0; k0 < h; k0 += blockDim.x) {
            const int64_t k = k0 + threadIdx.x;
            const double a = k < h ? __dadd_rn(ch[2 * k], ch[2 * k + 1]) : 0.0;
            __syncthreads();
            if (k < h) ch[k] = a;
            __syncthreads();
        }
        if (w & 1) {
            if (threadIdx.x == 0) ch[h] = ch[w - 1];
            __syncthreads();
        }
        w = h + (w & 1);
    }
    if (threadIdx.x == 0) *out = m ? ch[0] : 0.0;
}

// Normalise both weight sets, form phi2, and set the start (identity or the
// staged table rounded to the lattice).
__global__ void k2_scale_init(G2 g, double* __restrict__ px, double* __restrict__ p1,
                              double* __restrict__ phi2, const double* __restrict__ sums,
                              int64_t* __restrict__ nu, const double* __restrict__ table,
                              int from_table) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = g.n_x * g.n_x;
    if (i < n) {
        px[i] = __ddiv_rn(px[i], sums[0]);
        for (int k = 0; k < 2; ++k) {
            if (from_table) {
                const double v = __dmul_rn(__ddiv_rn(table[2 * i + k], g.delta), (double)g.one);
                nu[2 * i + k] = (int64_t)llround(v);
            } else {
                nu[2 * i + k] = ((k == 0 ? i / g.n_x : i % g.n_x) - g.hx) * g.one;
            }
        }
    }
    if (i < g.n_w * g.n_w) {
        const int64_t c = i / g.n_w, d = i % g.n_w;
        phi2[i] = __dmul_rn(__ddiv_rn(p1[c], sums[1]), __ddiv_rn(p1[d], sums[1]));
    }
}

// The staged table of controller values rounded to the lattice into nu.
__global__ void k2_table(G2 g, const double* __restrict__ table, int64_t* __restrict__ nu) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * g.n_x * g.n_x) return;
    nu[i] = (int64_t)llround(__dmul_rn(__ddiv_rn(table[i], g.delta), (double)g.one));
}

inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

const char* make_g2(const ucp2_params& p, G2* g) {
    *g = G2{};
    if (!(p.k > 0.0) || !(p.sigma > 0.0) || !(p.delta > 0.0)) return "k, sigma and delta must be > 0";
    auto steps = [&](double half, int64_t* out) {
        const double r = half / p.delta, n = floor(r + 0.5);
        if (!(n >= 0.0) || fabs(r - n) > 1e-9 * (n > 1.0 ? n : 1.0)) return false;
        *out = (int64_t)n;
        return true;
    };
    if (!steps(p.x_half, &g->hx) || !steps(p.w_half, &g->hw) || !steps(p.y_half, &g->hy) ||
        !steps(p.cand_half, &g->hr))
        return "half widths must be multiples of delta";
    if (p.n_coarse < 2 || p.n_coarse > 64) return "n_coarse must be in 2..64";
    if (p.n_levels < 0 || p.n_levels > 40) return "n_levels must be in 0..40";
    if (p.n_nbr < 0 || p.n_nbr > 8) return "n_nbr must be in 0..8";
    if (p.reserved != 0) return "reserved must be 0";
    g->k = p.k;
    g->kk = p.k * p.k;
    g->sigma = p.sigma;
    g->delta = p.delta;
    g->n_x = 2 * g->hx + 1;
    g->n_w = 2 * g->hw + 1;
    g->n_y = 2 * g->hy + 1;
    if (g->n_x > 441 || g->n_y > 2049 || g->n_w > 1025)
        return "grids too large (n_x <= 441, n_y <= 2049, n_w <= 1025 per axis)";
    g->shift = p.n_levels;
    g->one = (int64_t)1 << g->shift;
    const int64_t nc1 = p.n_coarse - 1, c = (g->hr + nc1 - 1) / nc1;
    g->q = 2 * (c < 1 ? 1 : c);
    const int64_t side = 2 * (int64_t)p.n_nbr + 1;
    g->n_cand = side * side + (int64_t)p.n_coarse * p.n_coarse + 8 * (int64_t)p.n_levels;
    g->n_coarse = p.n_coarse;
    g->n_levels = p.n_levels;
    g->n_nbr = p.n_nbr;
    const double vmax = (double)(g->hr + g->q + g->hx + g->hy + g->hw) * (double)g->one;
    if (!(vmax < 4.0e15)) return "lattice indices would overflow";
    return nullptr;
}

void launch2_setup(const G2& g, Dev2& d, int from_table, cudaStream_t s) {
    const int64_t n = g.n_x * g.n_x, big = n > g.n_w * g.n_w ? n : g.n_w * g.n_w;
    k2_exps<<<nblk(n > g.n_w ? n : g.n_w, 256), 256, 0, s>>>(g, d.px, d.phi1);
    k2_fixed_sum<<<1, 1024, 8 * sum_chunks(n), s>>>(d.px, n, d.scratch);
    k2_fixed_sum<<<1, 1024, 8 * sum_chunks(g.n_w), s>>>(d.phi1, g.n_w, d.scratch + 1);
    k2_scale_init<<<nblk(big, 256), 256, 0, s>>>(g, d.px, d.phi1, d.phi2, d.scratch, d.nu[0],
                                                 d.table, from_table);
}

void launch2_sweep(const G2& g, Dev2& d, int cur, cudaStream_t s) {
    const int64_t n = g.n_x * g.n_x;
    k2_search<<<nblk(32 * n, kSearch2T), kSearch2T, 0, s>>>(g, d.phi2, d.U, d.nu[cur],
                                                            d.nu[cur ^ 1], d.idx);
}

void launch2_mmse(const G2& g, Dev2& d, int buf, cudaStream_t s) {
    k2_mmse<<<nblk(g.n_y * g.n_y, 128), 128, 0, s>>>(g, d.nu[buf], d.U);
}

void launch2_J(const G2& g, Dev2& d, int buf, double* out, cudaStream_t s) {
    k2_costs<<<nblk(g.n_x * g.n_x, 128), 128, 0, s>>>(g, d.phi2, d.U, d.nu[buf], d.terms);
    k2_J<<<1, 32, 0, s>>>(g, d.px, d.terms, out);
}

void launch2_table(const G2& g, Dev2& d, int buf, cudaStream_t s) {
    k2_table<<<nblk(2 * g.n_x * g.n_x, 256), 256, 0, s>>>(g, d.table, d.nu[buf]);
}

}  // namespace ucp
