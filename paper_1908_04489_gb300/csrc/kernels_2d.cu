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

#include "df.cuh"
#include "fixed_sum.cuh"
#include "ucp_2d.h"
#include "ucp_runtime.h"

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

// Where the taps of S(u) at the lattice pair (nu1, nu2) read the u1 table:
// the cell of u (floor division), the fractions, the first tap's cell.
struct TapBase {
    int64_t jb1, jb2;
    double t1, t2, u1, u2;
};
__device__ __forceinline__ TapBase tap_base(const G2& g, int64_t nu1, int64_t nu2) {
    TapBase b;
    const int64_t c1 = nu1 >> g.shift, c2 = nu2 >> g.shift;   // floor division
    b.t1 = __dmul_rn((double)(nu1 - (c1 << g.shift)), inv_one2(g));
    b.t2 = __dmul_rn((double)(nu2 - (c2 << g.shift)), inv_one2(g));
    b.jb1 = c1 - g.hw + g.hy;
    b.jb2 = c2 - g.hw + g.hy;
    b.u1 = val2(g, nu1);
    b.u2 = val2(g, nu2);
    return b;
}
// Term (c, d) of S: phi_c phi_d |u - U^(u + w_cd)|^2.
__device__ __forceinline__ double tap2(const G2& g, const double* __restrict__ phi2,
                                       const double* __restrict__ U, const TapBase& b,
                                       int64_t c, int64_t d) {
    const double e1 = __dsub_rn(b.u1, bilerp2(g, U, 0, b.jb1 + c, b.jb2 + d, b.t1, b.t2));
    const double e2 = __dsub_rn(b.u2, bilerp2(g, U, 1, b.jb1 + c, b.jb2 + d, b.t1, b.t2));
    return __dmul_rn(phi2[c * g.n_w + d], __dadd_rn(__dmul_rn(e1, e1), __dmul_rn(e2, e2)));
}

// S(u) at the lattice pair (nu1, nu2): taps in row-major order, the fixed sum.
__device__ double S2d(const G2& g, const double* __restrict__ phi2,
                      const double* __restrict__ U, int64_t nu1, int64_t nu2) {
    const TapBase b = tap_base(g, nu1, nu2);
    const int64_t m = g.n_w;
    FixedSum acc;
    for (int64_t c = 0; c < m; ++c)
        for (int64_t d = 0; d < m; ++d) acc.add(tap2(g, phi2, U, b, c, d));
    return acc.result();
}

// k^2 |u - x|^2, the first part of the marginal cost, at x = (xa, xb).
__device__ __forceinline__ double kterm2x(const G2& g, double xa, double xb, int64_t nu1,
                                          int64_t nu2) {
    const double d1 = __dsub_rn(val2(g, nu1), xa);
    const double d2 = __dsub_rn(val2(g, nu2), xb);
    return __dmul_rn(g.kk, __dadd_rn(__dmul_rn(d1, d1), __dmul_rn(d2, d2)));
}
__device__ __forceinline__ double kterm2(const G2& g, int64_t i, int64_t nu1, int64_t nu2) {
    return kterm2x(g, grid2(g, i / g.n_x, g.hx), grid2(g, i % g.n_x, g.hx), nu1, nu2);
}

// Per-point constants of the search: grid coordinates and position.
struct Pt2 {
    int64_t i;
    int32_t a, b;
    double xa, xb;
    dfloat xa_d, xb_d;
};
__device__ __forceinline__ Pt2 make_pt2(const G2& g, int64_t i) {
    Pt2 q;
    q.i = i;
    q.a = (int32_t)(i / g.n_x);
    q.b = (int32_t)(i - (int64_t)q.a * g.n_x);
    q.xa = grid2(g, q.a, g.hx);
    q.xb = grid2(g, q.b, g.hx);
    q.xa_d = df_from_double(q.xa);
    q.xb_d = df_from_double(q.xb);
    return q;
}

__device__ __forceinline__ double cost2d(const G2& g, const double* __restrict__ phi2,
                                         const double* __restrict__ U, int64_t i,
                                         int64_t nu1, int64_t nu2) {
    return __dadd_rn(kterm2(g, i, nu1, nu2), S2d(g, phi2, U, nu1, nu2));
}

__device__ __forceinline__ bool before2(double ga, int32_t pa, double gb, int32_t pb) {
    return ga < gb || (ga == gb && pa < pb);
}

// Candidate p of stage 0 with the point's constants (32-bit index arithmetic).
__device__ __forceinline__ void stage0_cand_pt(const G2& g, const int64_t* __restrict__ nu_pre,
                                               const Pt2& q, int p, int64_t& n1, int64_t& n2) {
    const int r = g.n_nbr, side = 2 * r + 1, win = side * side;
    if (p == 0) {
        n1 = nu_pre[2 * q.i];
        n2 = nu_pre[2 * q.i + 1];
        return;
    }
    if (p < win) {
        const int k0 = p - 1, centre = r * side + r;
        const int k = k0 < centre ? k0 : k0 + 1;          // the window, centre skipped
        const int a = q.a + k / side - r, b = q.b + k % side - r;
        const int nx = (int)g.n_x;
        const int64_t j = (a < 0 || a >= nx || b < 0 || b >= nx) ? q.i : (int64_t)a * nx + b;
        n1 = nu_pre[2 * j];
        n2 = nu_pre[2 * j + 1];
        return;
    }
    const int ci = p - win, nc = g.n_coarse;
    const int64_t hq = g.q / 2;
    n1 = (int64_t)(2 * (ci / nc) - (nc - 1)) * hq * g.one;
    n2 = (int64_t)(2 * (ci % nc) - (nc - 1)) * hq * g.one;
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

// u1 step at target t directly: the exponents' minimum over the sources,
// then the two numerators and the denominator in source order.
__device__ void mmse_direct(const G2& g, const int64_t* __restrict__ nu, int64_t t,
                            double* __restrict__ U) {
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

// u1 step, one thread per target t (the direct form).
__global__ void __launch_bounds__(128) k2_mmse(G2 g, const int64_t* __restrict__ nu,
                                               double* __restrict__ U) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < g.n_y * g.n_y) mmse_direct(g, nu, t, U);
}

// ---- factorised u1 step -------------------------------------------------------
//
// The exponent of source i at target y splits over the axes,
//   E_i(y) = P_i + Q_i(y_1) + R_i(y_2),  P_i = |x_i|^2 / (2 sigma^2),
//   Q_i(y_1) = (y_1 - f_i1)^2 / 2,  R_i(y_2) = (y_2 - f_i2)^2 / 2,
// so exp(-(E_i - e)) with e = min_i (P_i + Q_i(y_1)) + min_i R_i(y_2) is the
// product a_i(y_1) b_i(y_2) of per-axis factors (the prior folded into a).
// The weights differ from exp(-(E_i - min_i E_i)) by one factor per target,
// which cancels in the ratio; the three sums over sources are then
// GEMM-shaped (n_y x n_y targets, n_x^2 sources) and run split over source
// ranges, the partial sums added in split order.  The factors are at most 1
// and terms below FP32's range are lost, so a target whose denominator (that
// cancelled factor, at least) falls below 2^-60 is recomputed in the direct
// form; elsewhere the lost terms are below 2^-50 of the denominator.

// Per source: fv[2 i + q] = f_iq and fv[2 N + i] = P_i.
__device__ __forceinline__ double half_sq(double y, double f) {
    const double d = y - f;
    return 0.5 * (d * d);
}
__device__ __forceinline__ double prior_expo(const G2& g, int64_t i) {
    const double xa = grid2(g, i / g.n_x, g.hx), xb = grid2(g, i % g.n_x, g.hx);
    return (xa * xa + xb * xb) / (2.0 * g.sigma * g.sigma);
}
__global__ void __launch_bounds__(256) k2_u1_sources(G2 g, const int64_t* __restrict__ nu,
                                                     double* __restrict__ fv) {
    const int64_t n = g.n_x * g.n_x;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    fv[2 * i] = val2(g, nu[2 * i]);
    fv[2 * i + 1] = val2(g, nu[2 * i + 1]);
    fv[2 * n + i] = prior_expo(g, i);
}

// The axis shifts: mins[j] = min_i (P_i + Q_i(y_j)) (the prior folded into
// axis 1, which keeps the joint minimum closer to the sum of the shifts) and
// mins[n_y + j] = min_i R_i(y_j); one block each.
__global__ void __launch_bounds__(256) k2_u1_mins(G2 g, const double* __restrict__ fv,
                                                  double* __restrict__ mins) {
    __shared__ double red[256];
    const int64_t b = blockIdx.x, n = g.n_x * g.n_x;
    const int q = b < g.n_y ? 0 : 1;
    const double y = grid2(g, b - q * g.n_y, g.hy);
    double m = INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        m = fmin(m, (q == 0 ? fv[2 * n + i] : 0.0) + half_sq(y, fv[2 * i + q]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) mins[b] = red[0];
}

// Factor tables, target-major (entry j N + i, N = n_x^2 sources):
//   fa = exp(-(P_i + Q_i(y_j) - mins[j])),  fb = exp(-(R_i(y_j) - mins[n_y + j])),
// both at most 1, formed in FP64 and kept as double-float pairs (hi, lo) for
// the sums and in FP64 for the targets whose factor leaves FP32's range.
__global__ void __launch_bounds__(256) k2_u1_factors(G2 g, const double* __restrict__ mins,
                                                     const double* __restrict__ fv,
                                                     float2* __restrict__ fa,
                                                     float2* __restrict__ fb,
                                                     double* __restrict__ fa64,
                                                     double* __restrict__ fb64) {
    const int64_t n = g.n_x * g.n_x;
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n * g.n_y) return;
    const int64_t j = id / n, i = id % n;
    const double y = grid2(g, j, g.hy);
    const double va = exp(-((fv[2 * n + i] + half_sq(y, fv[2 * i])) - mins[j]));
    const double vb = exp(-(half_sq(y, fv[2 * i + 1]) - mins[g.n_y + j]));
    const dfloat a = df_from_double(va), b = df_from_double(vb);
    fa[id] = make_float2(a.hi, a.lo);
    fb[id] = make_float2(b.hi, b.lo);
    fa64[id] = va;
    fb64[id] = vb;
}

// Partial sums of one split of the sources for a 32 x 32 tile of targets in
// double-float arithmetic on the FP32 pipe: 256 threads, each a 2 x 2 block
// of targets (rows 2 ty + r, columns tx + 16 c; a warp holds four whole
// rows), 32 sources per shared-memory stage.  Each stage is summed afresh (products kept as
// unnormalised pairs, accumulation normalised per term) and then added to
// the running sums with the accurate double-float addition, so a split of K
// sources carries a relative error of about (32 + K / 32) 2^-47 of its sum
// of magnitudes.  Stages that cannot matter on the tile are skipped.
constexpr int kU1Tile = 32, kU1Stage = 32;
constexpr unsigned kFull2 = 0xffffffffu;
__global__ void __launch_bounds__(256) k2_u1_sums(G2 g, const float2* __restrict__ fa,
                                                  const float2* __restrict__ fb,
                                                  const double* __restrict__ fv,
                                                  int64_t split_len, double* __restrict__ part,
                                                  unsigned long long* __restrict__ live_pairs) {
    __shared__ float2 sa[kU1Stage][kU1Tile + 1], sb[kU1Stage][kU1Tile + 1], sf[kU1Stage][2];
    __shared__ unsigned wmax[2][8];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t ny = g.n_y, n = g.n_x * g.n_x;
    const int64_t j1_0 = (int64_t)blockIdx.y * kU1Tile, j2_0 = (int64_t)blockIdx.x * kU1Tile;
    const int64_t i_lo = (int64_t)blockIdx.z * split_len;
    const int64_t i_hi = min(i_lo + split_len, n);
    dfloat D[2][2], N1[2][2], N2[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) D[r][c] = N1[r][c] = N2[r][c] = dfloat{0.0f, 0.0f};
    for (int64_t i0 = i_lo; i0 < i_hi; i0 += kU1Stage) {
        unsigned ma = 0u, mb = 0u;   // bit patterns of the largest factors (>= 0)
        for (int k = threadIdx.x; k < kU1Stage * kU1Tile; k += 256) {
            const int sj = k / kU1Stage, si = k % kU1Stage;   // consecutive sources
            const int64_t i = i0 + si;
            const bool ok = i < i_hi;
            const float2 va = ok && j1_0 + sj < ny ? fa[(j1_0 + sj) * n + i] : make_float2(0.f, 0.f);
            const float2 vb = ok && j2_0 + sj < ny ? fb[(j2_0 + sj) * n + i] : make_float2(0.f, 0.f);
            sa[si][sj] = va;
            sb[si][sj] = vb;
            ma = max(ma, __float_as_uint(va.x));
            mb = max(mb, __float_as_uint(vb.x));
        }
        if (threadIdx.x < 2 * kU1Stage) {
            const int si = threadIdx.x >> 1, q = threadIdx.x & 1;
            const int64_t i = i0 + si;
            const dfloat f = df_from_double(i < i_hi ? fv[2 * i + q] : 0.0);
            sf[si][q] = make_float2(f.hi, f.lo);
        }
        // A stage whose largest axis-1 factor times largest axis-2 factor on
        // this tile is below 2^-126 adds less than N 2^-126 to any sum: at most
        // 2^-48 of a denominator that stays on this path (>= 2^-60).
        ma = __reduce_max_sync(kFull2, ma);
        mb = __reduce_max_sync(kFull2, mb);
        if ((threadIdx.x & 31) == 0) {
            wmax[0][threadIdx.x >> 5] = ma;
            wmax[1][threadIdx.x >> 5] = mb;
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            ma = max(ma, wmax[0][w]);
            mb = max(mb, wmax[1][w]);
        }
        const bool live = __uint_as_float(ma) * __uint_as_float(mb) >= 0x1p-126f;
        if (!live) {
            __syncthreads();
            continue;
        }
        // The same test per warp: its four target rows' largest axis-1 factor
        // times the tile's largest axis-2 factor.  The flag is warp-uniform and
        // every warp reaches the stage's closing barrier either way.
        bool warp_live;
        {
            const int lane = threadIdx.x & 31, r0 = 4 * (threadIdx.x >> 5);
            unsigned wa = 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) wa = max(wa, __float_as_uint(sa[lane][r0 + k].x));
            wa = __reduce_max_sync(kFull2, wa);
            warp_live = __uint_as_float(wa) * __uint_as_float(mb) >= 0x1p-126f;
            if (warp_live && lane == 0)
                atomicAdd(live_pairs, (unsigned long long)(kU1Stage * 4 * kU1Tile));
        }
        if (warp_live) {
            dfloat d[2][2], m1[2][2], m2[2][2];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c) d[r][c] = m1[r][c] = m2[r][c] = dfloat{0.0f, 0.0f};
#pragma unroll 2
            for (int si = 0; si < kU1Stage; ++si) {
                dfloat a[2], b[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float2 v = sa[si][2 * ty + r];
                    a[r] = dfloat{v.x, v.y};
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float2 v = sb[si][tx + 16 * c];
                    b[c] = dfloat{v.x, v.y};
                }
                const float2 f1 = sf[si][0], f2 = sf[si][1];
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        float p, e, q, qe;
                        df_mul_raw(a[r], b[c], p, e);
                        d[r][c] = df_acc(d[r][c], p, e);
                        df_mul_raw(dfloat{p, e}, dfloat{f1.x, f1.y}, q, qe);
                        m1[r][c] = df_acc(m1[r][c], q, qe);
                        df_mul_raw(dfloat{p, e}, dfloat{f2.x, f2.y}, q, qe);
                        m2[r][c] = df_acc(m2[r][c], q, qe);
                    }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    D[r][c] = df_add_acc(D[r][c], d[r][c]);
                    N1[r][c] = df_add_acc(N1[r][c], m1[r][c]);
                    N2[r][c] = df_add_acc(N2[r][c], m2[r][c]);
                }
        }   // warp_live
        __syncthreads();
    }
    const int64_t plane = ny * ny;
    double* out = part + (int64_t)blockIdx.z * 3 * plane;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int64_t j1 = j1_0 + 2 * ty + r, j2 = j2_0 + tx + 16 * c;
            if (j1 < ny && j2 < ny) {
                const int64_t t = j1 * ny + j2;
                out[t] = df_to_double(D[r][c]);
                out[plane + t] = df_to_double(N1[r][c]);
                out[2 * plane + t] = df_to_double(N2[r][c]);
            }
        }
}

// U = numerators / denominator with the splits added in order; targets
// whose denominator is below 2^-60 are listed for the FP64 pass.
__global__ void __launch_bounds__(128) k2_u1_finish(G2 g, const double* __restrict__ part,
                                                    int splits, double* __restrict__ U,
                                                    int32_t* __restrict__ list) {
    const int64_t plane = g.n_y * g.n_y;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= plane) return;
    double den = 0.0, a1 = 0.0, a2 = 0.0;
    for (int s = 0; s < splits; ++s) {
        const double* p = part + (int64_t)s * 3 * plane;
        den += p[t];
        a1 += p[plane + t];
        a2 += p[2 * plane + t];
    }
    if (den >= 0x1p-60) {
        U[2 * t] = a1 / den;
        U[2 * t + 1] = a2 / den;
    } else {
        list[1 + atomicAdd(list, 1)] = (int32_t)t;
    }
}

// The listed targets in FP64, one warp each: lane l sums sources l, l + 32,
// ... of the FP64 factor tables, then a fixed reduction tree.  FP64's range
// keeps every term above 2^-50 of the denominator while that is at least
// 2^-957; below that (a factor gap beyond ~660) the direct form runs.
__global__ void __launch_bounds__(128) k2_u1_wide(G2 g, const int64_t* __restrict__ nu,
                                                  const double* __restrict__ fa64,
                                                  const double* __restrict__ fb64,
                                                  const double* __restrict__ fv,
                                                  const int32_t* __restrict__ list,
                                                  double* __restrict__ U) {
    const int lane = threadIdx.x & 31;
    const int64_t n = g.n_x * g.n_x, count = list[0];
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; w < count;
         w += warps) {
        const int64_t t = list[1 + w], j1 = t / g.n_y, j2 = t % g.n_y;
        const double* a = fa64 + j1 * n;
        const double* b = fb64 + j2 * n;
        double den = 0.0, s1 = 0.0, s2 = 0.0;
        for (int64_t i = lane; i < n; i += 32) {
            const double v = a[i] * b[i];
            den += v;
            s1 += v * fv[2 * i];
            s2 += v * fv[2 * i + 1];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            den += __shfl_xor_sync(0xffffffffu, den, off);
            s1 += __shfl_xor_sync(0xffffffffu, s1, off);
            s2 += __shfl_xor_sync(0xffffffffu, s2, off);
        }
        if (den >= 0x1p-957) {
            if (lane == 0) {
                U[2 * t] = s1 / den;
                U[2 * t + 1] = s2 / den;
            }
        } else if (lane == 0) {
            mmse_direct(g, nu, t, U);
        }
    }
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

// out = scale x the sum of v[0..n) in the fixed order (32-term chunks left to
// right, then pairwise by levels): one block, chunk sums in shared memory,
// each level's additions spread over the block.
__global__ void k2_fixed_sum(const double* __restrict__ v, int64_t n, double scale,
                             double* __restrict__ out) {
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
    if (threadIdx.x == 0) *out = __dmul_rn(scale, m ? ch[0] : 0.0);
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

// ---- screened search --------------------------------------------------------
//
// With U^ bilinear, S(u) = W |u|^2 - 2 u . sum_k a_k A(j + o_k)
//                          + sum_kl a_k a_l C_{o_l - o_k}(j + o_k),
// j the first tap's cell, o_k in {(0,0), (0,1), (1,0), (1,1)} the cell's
// corners with bilinear weights a_k, W = sum_cd phi_c phi_d, and
//   A_q(j) = sum_cd phi_c phi_d U_q(j + (c, d))               (q = 1, 2),
//   C_e(j) = sum_cd phi_c phi_d <U(j + (c, d)), U(j + (c, d) + e)>,
// e in {(0,0), (0,1), (1,0), (1,1), (1,-1)}, U clamped beyond its grid.  Every
// table is constant for j below -n_w - 1 or above n_y on an axis (all its
// taps read the clamped edge there), so corner indices are clamped to that
// range.  Slots of a cell: A_1, A_2, C_00, C_01, C_10, C_11, C_1m, unused.

// Umax = max |U| (every block's maximum folded in by an atomic maximum on
// the bit patterns, which order like the non-negative doubles; out[0] is
// zeroed before) and W = (sum_c phi_c)^2 (block 0).
__global__ void __launch_bounds__(256) k2_tab_consts(G2 g, const double* __restrict__ U,
                                                     const double* __restrict__ phin,
                                                     double* __restrict__ out) {
    __shared__ double red[256];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    red[threadIdx.x] = k < 2 * g.n_y * g.n_y ? fabs(U[k]) : 0.0;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicMax(reinterpret_cast<unsigned long long*>(out),
                  (unsigned long long)__double_as_longlong(red[0]));
        if (blockIdx.x == 0) {
            double w = 0.0;
            for (int64_t c = 0; c < g.n_w; ++c) w += phin[c];
            out[1] = w * w;
        }
    }
}

// Row pass: H_f(r, a2) = sum_d phi_d F_f(J1, J2 + d), J1 = tab_lo + r,
// J2 = tab_lo + a2, with the fields F = U_1, U_2 and <U(J), U(J + e)>.
__global__ void __launch_bounds__(256) k2_tab_rows(G2 g, const double* __restrict__ U,
                                                   const double* __restrict__ phin,
                                                   double* __restrict__ H) {
    const int64_t L = g.tab_n, plane = g.ext_n * L;
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= plane) return;
    const int64_t J1 = g.tab_lo + id / L, J2 = g.tab_lo + id % L, n = g.n_y;
    const int64_t ra = clampy(g, J1) * n, rb = clampy(g, J1 + 1) * n;
    double acc[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t d = 0; d < g.n_w; ++d) {
        const int64_t ca = clampy(g, J2 + d), cb = clampy(g, J2 + d + 1),
                      cm = clampy(g, J2 + d - 1);
        const double2 u = *reinterpret_cast<const double2*>(U + 2 * (ra + ca));
        const double2 r = *reinterpret_cast<const double2*>(U + 2 * (ra + cb));   // e = (0, 1)
        const double2 v = *reinterpret_cast<const double2*>(U + 2 * (rb + ca));   // e = (1, 0)
        const double2 q = *reinterpret_cast<const double2*>(U + 2 * (rb + cb));   // e = (1, 1)
        const double2 m = *reinterpret_cast<const double2*>(U + 2 * (rb + cm));   // e = (1, -1)
        const double w = phin[d];
        acc[0] += w * u.x;
        acc[1] += w * u.y;
        acc[2] += w * (u.x * u.x + u.y * u.y);
        acc[3] += w * (u.x * r.x + u.y * r.y);
        acc[4] += w * (u.x * v.x + u.y * v.y);
        acc[5] += w * (u.x * q.x + u.y * q.y);
        acc[6] += w * (u.x * m.x + u.y * m.y);
    }
#pragma unroll
    for (int f = 0; f < 7; ++f) H[f * plane + id] = acc[f];
}

// Column pass: tab(a1, a2) = sum_c phi_c H(a1 + c, a2), 8 slots per cell.
__global__ void __launch_bounds__(256) k2_tab_cols(G2 g, const double* __restrict__ H,
                                                   const double* __restrict__ phin,
                                                   double* __restrict__ tab,
                                                   float2* __restrict__ tabf) {
    const int64_t L = g.tab_n, plane = g.ext_n * L;
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= L * L) return;
    const int64_t a1 = id / L, a2 = id % L;
    double acc[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t c = 0; c < g.n_w; ++c) {
        const double w = phin[c];
        const double* h = H + (a1 + c) * L + a2;
#pragma unroll
        for (int f = 0; f < 7; ++f) acc[f] += w * h[f * plane];
    }
    double2* o = reinterpret_cast<double2*>(tab + 8 * id);
    o[0] = make_double2(acc[0], acc[1]);
    o[1] = make_double2(acc[2], acc[3]);
    o[2] = make_double2(acc[4], acc[5]);
    o[3] = make_double2(acc[6], 0.0);
    float4* of = reinterpret_cast<float4*>(tabf + 8 * id);
    dfloat v[8];
#pragma unroll
    for (int f = 0; f < 7; ++f) v[f] = df_from_double(acc[f]);
    v[7] = dfloat{0.0f, 0.0f};
#pragma unroll
    for (int f = 0; f < 4; ++f)
        of[f] = make_float4(v[2 * f].hi, v[2 * f].lo, v[2 * f + 1].hi, v[2 * f + 1].lo);
}

__device__ __forceinline__ int64_t tcell(const G2& g, int64_t j) {
    const int64_t hi = g.tab_lo + g.tab_n - 1;
    return (j < g.tab_lo ? g.tab_lo : (j > hi ? hi : j)) - g.tab_lo;
}

// Table cost of candidate (nu1, nu2) at x0 point i and the bound eb on its
// distance from the exact fixed-order cost cost2d.
__device__ __forceinline__ void tab_cost(const G2& g, const double* __restrict__ tab, double um,
                                         double W, const Pt2& pt, int64_t nu1, int64_t nu2,
                                         double& gt, double& eb) {
    const TapBase b = tap_base(g, nu1, nu2);
    const int64_t L = g.tab_n;
    const int64_t a1 = tcell(g, b.jb1), a1p = tcell(g, b.jb1 + 1);
    const int64_t a2 = tcell(g, b.jb2), a2p = tcell(g, b.jb2 + 1);
    const double* P00 = tab + 8 * (a1 * L + a2);
    const double* P01 = tab + 8 * (a1 * L + a2p);
    const double* P10 = tab + 8 * (a1p * L + a2);
    const double* P11 = tab + 8 * (a1p * L + a2p);
    const double s1 = 1.0 - b.t1, s2 = 1.0 - b.t2;
    const double w00 = s1 * s2, w01 = s1 * b.t2, w10 = b.t1 * s2, w11 = b.t1 * b.t2;
    const double A1 = w00 * P00[0] + w01 * P01[0] + w10 * P10[0] + w11 * P11[0];
    const double A2 = w00 * P00[1] + w01 * P01[1] + w10 * P10[1] + w11 * P11[1];
    const double Cd = w00 * w00 * P00[2] + w01 * w01 * P01[2] + w10 * w10 * P10[2] +
                      w11 * w11 * P11[2];
    const double Cx = w00 * w01 * P00[3] + w00 * w10 * P00[4] + w00 * w11 * P00[5] +
                      w01 * w10 * P01[6] + w01 * w11 * P01[4] + w10 * w11 * P10[3];
    const double uu = b.u1 * b.u1 + b.u2 * b.u2;
    const double S = W * uu - 2.0 * (b.u1 * A1 + b.u2 * A2) + Cd + 2.0 * Cx;
    gt = kterm2x(g, pt.xa, pt.xb, nu1, nu2) + S;
    const double M = uu + 2.0 * (fabs(b.u1) + fabs(b.u2)) * um + 2.0 * um * um;
    eb = g.eps_k * (M + fabs(gt));
}

// The table cost in double-float arithmetic on the FP32 pipe, with the
// bound eps_df (M + |g|).  The bilinear weights are exact pairs (the
// fractions have at most 24 bits); products are accumulated unnormalised
// into normalised sums.  False (nothing computed) when a lattice index is
// beyond 2^44, where the pair conversion is not exact.
__device__ __forceinline__ dfloat df_dot_add(dfloat acc, dfloat a, dfloat b) {
    float p, e;
    df_mul_raw(a, b, p, e);
    return df_acc(acc, p, e);
}
__device__ __forceinline__ bool tab_cost_df(const G2& g, const float2* __restrict__ tabf,
                                            float um, dfloat W, const Pt2& pt, int64_t nu1,
                                            int64_t nu2, dfloat& lo, dfloat& hi) {
    const int64_t lim = (int64_t)1 << 44;
    if (nu1 >= lim || nu1 <= -lim || nu2 >= lim || nu2 <= -lim) return false;
    const int64_t c1 = nu1 >> g.shift, c2 = nu2 >> g.shift;
    const float t1 = __fmul_rn(__int2float_rn((int)(nu1 - (c1 << g.shift))), g.inv_one_f);
    const float t2 = __fmul_rn(__int2float_rn((int)(nu2 - (c2 << g.shift))), g.inv_one_f);
    const float s1 = __fsub_rn(1.0f, t1), s2 = __fsub_rn(1.0f, t2);   // exact
    auto exact_prod = [](float a, float b) {
        const float p = __fmul_rn(a, b);
        return dfloat{p, __fmaf_rn(a, b, -p)};
    };
    const dfloat w00 = exact_prod(s1, s2), w01 = exact_prod(s1, t2);
    const dfloat w10 = exact_prod(t1, s2), w11 = exact_prod(t1, t2);
    const int64_t L = g.tab_n, jb1 = c1 - g.hw + g.hy, jb2 = c2 - g.hw + g.hy;
    const int64_t a1 = tcell(g, jb1), a1p = tcell(g, jb1 + 1);
    const int64_t a2 = tcell(g, jb2), a2p = tcell(g, jb2 + 1);
    const float2* P00 = tabf + 8 * (a1 * L + a2);
    const float2* P01 = tabf + 8 * (a1 * L + a2p);
    const float2* P10 = tabf + 8 * (a1p * L + a2);
    const float2* P11 = tabf + 8 * (a1p * L + a2p);
    auto T = [](const float2* P, int f) {
        const float2 v = P[f];
        return dfloat{v.x, v.y};
    };
    const dfloat z{0.0f, 0.0f};
    dfloat A1 = df_dot_add(z, w00, T(P00, 0));
    A1 = df_dot_add(A1, w01, T(P01, 0));
    A1 = df_dot_add(A1, w10, T(P10, 0));
    A1 = df_dot_add(A1, w11, T(P11, 0));
    dfloat A2 = df_dot_add(z, w00, T(P00, 1));
    A2 = df_dot_add(A2, w01, T(P01, 1));
    A2 = df_dot_add(A2, w10, T(P10, 1));
    A2 = df_dot_add(A2, w11, T(P11, 1));
    dfloat C = df_dot_add(z, df_mul(w00, w00), T(P00, 2));
    C = df_dot_add(C, df_mul(w01, w01), T(P01, 2));
    C = df_dot_add(C, df_mul(w10, w10), T(P10, 2));
    C = df_dot_add(C, df_mul(w11, w11), T(P11, 2));
    dfloat X = df_dot_add(z, df_mul(w00, w01), T(P00, 3));
    X = df_dot_add(X, df_mul(w00, w10), T(P00, 4));
    X = df_dot_add(X, df_mul(w00, w11), T(P00, 5));
    X = df_dot_add(X, df_mul(w01, w10), T(P01, 6));
    X = df_dot_add(X, df_mul(w01, w11), T(P01, 4));
    X = df_dot_add(X, df_mul(w10, w11), T(P10, 3));
    const dfloat us{g.us_hi, g.us_lo};
    const dfloat u1 = df_mul(df_from_i64(nu1), us), u2 = df_mul(df_from_i64(nu2), us);
    const dfloat uu = df_dot_add(df_mul(u1, u1), u2, u2);
    dfloat S = df_mul(W, uu);
    S = df_dot_add(S, dfloat{-2.0f * u1.hi, -2.0f * u1.lo}, A1);
    S = df_dot_add(S, dfloat{-2.0f * u2.hi, -2.0f * u2.lo}, A2);
    S = df_add(S, C);
    S = df_add(S, dfloat{2.0f * X.hi, 2.0f * X.lo});
    const dfloat d1 = df_sub(u1, pt.xa_d), d2 = df_sub(u2, pt.xb_d);
    const dfloat kt = df_mul(df_dot_add(df_mul(d1, d1), d2, d2), dfloat{g.kk_hi, g.kk_lo});
    const dfloat gv = df_add(kt, S);
    // the bound in FP32 (eps_df rounded up, M and |g| to ~2^-21), widened by
    // 0.1%, which also covers the pair additions forming the interval's ends
    // (2^-47 |g| against eb >= 2^-37 M)
    const float ua = fabsf(u1.hi) + fabsf(u2.hi);
    const float M = uu.hi + 2.0f * ua * um + 2.0f * um * um;
    const float eb = g.eps_df_f * (M + fabsf(gv.hi)) * 1.001f;
    lo = df_add_f(gv, -eb);
    hi = df_add_f(gv, eb);
    return true;
}

constexpr unsigned kFull = 0xffffffffu;
constexpr int kExactCh = 512;   // chunk sums of one exact cost a warp keeps in shared memory

__device__ __forceinline__ dfloat warp_min_df(dfloat v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const dfloat o{__shfl_xor_sync(kFull, v.hi, off), __shfl_xor_sync(kFull, v.lo, off)};
        if (df_lt(o, v)) v = o;
    }
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

// The exact cost cost2d of (nu1, nu2) at point i, by the whole warp: lane l
// forms chunks l, l + 32, ... (each left to right, as FixedSum), then the
// chunk sums are paired level by level in shared memory.  Same double as
// cost2d.  Quadratures of more than kExactCh chunks run on lane 0.
__device__ double warp_exact(const G2& g, const double* __restrict__ phi2,
                             const double* __restrict__ U, int64_t i, int64_t nu1, int64_t nu2,
                             double* ch, int lane) {
    const int64_t T = g.n_w * g.n_w, m = sum_chunks(T);
    double S;
    if (m > kExactCh) {
        double v = 0.0;
        if (lane == 0) v = S2d(g, phi2, U, nu1, nu2);
        S = __shfl_sync(kFull, v, 0);
    } else {
        const TapBase b = tap_base(g, nu1, nu2);
        for (int64_t k = lane; k < m; k += 32) {
            const int64_t j0 = k * kSumChunk, e = min(j0 + kSumChunk, T);
            int64_t c = j0 / g.n_w, d = j0 % g.n_w;
            double a = 0.0;
            for (int64_t j = j0; j < e; ++j) {
                a = __dadd_rn(a, tap2(g, phi2, U, b, c, d));
                if (++d == g.n_w) {
                    d = 0;
                    ++c;
                }
            }
            ch[k] = a;
        }
        __syncwarp();
        for (int64_t w = m; w > 1;) {
            const int64_t h = w / 2;
            for (int64_t k0 = 0; k0 < h; k0 += 32) {
                const int64_t k = k0 + lane;
                const double a = k < h ? __dadd_rn(ch[2 * k], ch[2 * k + 1]) : 0.0;
                __syncwarp();
                if (k < h) ch[k] = a;
                __syncwarp();
            }
            if (w & 1) {
                if (lane == 0) ch[h] = ch[w - 1];
                __syncwarp();
            }
            w = h + (w & 1);
        }
        S = ch[0];
        __syncwarp();   // ch is reused by the next call
    }
    return __dadd_rn(kterm2(g, i, nu1, nu2), S);
}

// Resolution of one stage of the list: its contenders (table cost within the
// bound of the stage's best bound) offered in list order; the winner is the
// first with the least exact cost.  A value offered again is skipped (same
// exact cost, later position).  Exact costs are formed only once a second
// distinct value appears.  Warp-uniform except the seen list (lane k holds
// the k-th distinct value).
struct Stage2 {
    bool has = false, known = false;
    int64_t b1 = 0, b2 = 0;
    int32_t bp = 0;
    dfloat blo{0.f, 0.f}, bhi{0.f, 0.f};
    double bex = 0.0;
    int nseen = 0;
    int64_t s1 = 0, s2 = 0;

    __device__ void offer(const G2& g, const double* __restrict__ phi2,
                          const double* __restrict__ U, int64_t i, double* ch, int lane,
                          int64_t v1, int64_t v2, int32_t pos, dfloat vlo, dfloat vhi,
                          bool vknown, double vex) {
        if (__any_sync(kFull, lane < nseen && s1 == v1 && s2 == v2)) return;
        if (nseen < 32) {
            if (lane == nseen) {
                s1 = v1;
                s2 = v2;
            }
            ++nseen;
        }
        if (!has) {
            has = true;
            b1 = v1; b2 = v2; bp = pos; blo = vlo; bhi = vhi;
            known = vknown;
            bex = vex;
            return;
        }
        if (!known) {
            bex = warp_exact(g, phi2, U, i, b1, b2, ch, lane);
            known = true;
        }
        const double ex = vknown ? vex : warp_exact(g, phi2, U, i, v1, v2, ch, lane);
        if (ex < bex) {
            b1 = v1; b2 = v2; bp = pos; blo = vlo; bhi = vhi; bex = ex;
        }
    }
};

// One warp per x0 point, the list of k2_search with table costs: per stage
// the threshold min (gt + eb), then the contenders gt - eb <= threshold in
// list order (any other candidate's exact cost exceeds the stage minimum's).
__global__ void __launch_bounds__(kSearch2T) k2_search_scr(
    G2 g, const double* __restrict__ phi2, const double* __restrict__ U,
    const double* __restrict__ tab, const float2* __restrict__ tabf,
    const double* __restrict__ consts,
    const int64_t* __restrict__ nu_pre, int64_t* __restrict__ nu_out,
    int32_t* __restrict__ idx_out) {
    __shared__ double chs[kSearch2T / 32][kExactCh];
    const int lane = threadIdx.x & 31;
    double* ch = chs[threadIdx.x >> 5];
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (i >= g.n_x * g.n_x) return;   // the same for the warp
    const double um = consts[0], W = consts[1];
    const dfloat Wd = df_from_double(W);
    const float umf = __double2float_ru(um);
    const Pt2 pt = make_pt2(g, i);
    // The certified interval [g~ - eb, g~ + eb] of a candidate's exact cost as
    // double-float ends: from the double-float table cost where it applies,
    // else from the FP64 one (ends widened by 10%, far more than their
    // rounding to pairs).  Lexicographic comparison of normalised pairs is
    // exact, so the stage logic below is the FP64 one.
    auto cost = [&](int64_t n1, int64_t n2, dfloat& lo, dfloat& hi) {
        if (g.use_df && tab_cost_df(g, tabf, umf, Wd, pt, n1, n2, lo, hi)) return;
        double gt, eb;
        tab_cost(g, tab, um, W, pt, n1, n2, gt, eb);
        lo = df_from_double(gt - 1.1 * eb);
        hi = df_from_double(gt + 1.1 * eb);
    };
    const dfloat inf{FLT_MAX, 0.f};
    const int64_t side = 2 * (int64_t)g.n_nbr + 1;
    const int n0 = (int)(side * side + (int64_t)g.n_coarse * g.n_coarse);
    dfloat thr = inf;
    for (int p = lane; p < n0; p += 32) {
        int64_t n1, n2;
        dfloat lo, hi;
        stage0_cand_pt(g, nu_pre, pt, p, n1, n2);
        cost(n1, n2, lo, hi);
        if (df_lt(hi, thr)) thr = hi;
    }
    thr = warp_min_df(thr);
    Stage2 st;
    for (int base = 0; base < n0; base += 32) {
        const int p = base + lane;
        int64_t n1 = 0, n2 = 0;
        dfloat lo = inf, hi = inf;
        bool cont = false;
        if (p < n0) {
            stage0_cand_pt(g, nu_pre, pt, p, n1, n2);
            cost(n1, n2, lo, hi);
            cont = !df_lt(thr, lo);
        }
        unsigned mask = __ballot_sync(kFull, cont);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            st.offer(g, phi2, U, i, ch, lane, __shfl_sync(kFull, n1, src),
                     __shfl_sync(kFull, n2, src), base + src,
                     dfloat{__shfl_sync(kFull, lo.hi, src), __shfl_sync(kFull, lo.lo, src)},
                     dfloat{__shfl_sync(kFull, hi.hi, src), __shfl_sync(kFull, hi.lo, src)},
                     false, 0.0);
        }
    }
    int pos = n0;
    for (int lv = 1; lv <= g.n_levels; ++lv) {
        const int64_t h = g.q << (g.n_levels - lv);
        int64_t n1 = 0, n2 = 0;
        dfloat lo = inf, hi = inf;
        if (lane < 8) {
            const int k9 = lane < 4 ? lane : lane + 1;       // 3 x 3 window, centre skipped
            n1 = st.b1 + (int64_t)(k9 / 3 - 1) * h;
            n2 = st.b2 + (int64_t)(k9 % 3 - 1) * h;
            cost(n1, n2, lo, hi);
        }
        dfloat t = warp_min_df(hi);
        if (df_lt(st.bhi, t)) t = st.bhi;
        Stage2 nx;
        if (!df_lt(t, st.blo))
            nx.offer(g, phi2, U, i, ch, lane, st.b1, st.b2, st.bp, st.blo, st.bhi, st.known,
                     st.bex);
        unsigned mask = __ballot_sync(kFull, lane < 8 && !df_lt(t, lo));
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            nx.offer(g, phi2, U, i, ch, lane, __shfl_sync(kFull, n1, src),
                     __shfl_sync(kFull, n2, src), pos + src,
                     dfloat{__shfl_sync(kFull, lo.hi, src), __shfl_sync(kFull, lo.lo, src)},
                     dfloat{__shfl_sync(kFull, hi.hi, src), __shfl_sync(kFull, hi.lo, src)},
                     false, 0.0);
        }
        st = nx;
        pos += 8;
    }
    if (lane == 0) {
        nu_out[2 * i] = st.b1;
        nu_out[2 * i + 1] = st.b2;
        idx_out[i] = st.bp;
    }
}

// J's terms p_i g(f_i; x_i), one warp per point (the exact cost, the same
// double as cost2d).
__global__ void __launch_bounds__(kSearch2T) k2_J_terms(G2 g, const double* __restrict__ phi2,
                                                        const double* __restrict__ U,
                                                        const double* __restrict__ px,
                                                        const int64_t* __restrict__ nu,
                                                        double* __restrict__ terms) {
    __shared__ double chs[kSearch2T / 32][kExactCh];
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (i >= g.n_x * g.n_x) return;   // the same for the warp
    const double c = warp_exact(g, phi2, U, i, nu[2 * i], nu[2 * i + 1], chs[threadIdx.x >> 5],
                                lane);
    if (lane == 0) terms[i] = __dmul_rn(px[i], c);
}

// J's terms p_i g~(f_i; x_i) from the correlation tables (the screened
// mode): |g~ - g| <= eb_i, so J is within (1/2) sum_i p_i eb_i of the exact
// fixed-order J.
__global__ void __launch_bounds__(256) k2_J_terms_tab(G2 g, const double* __restrict__ tab,
                                                      const double* __restrict__ consts,
                                                      const double* __restrict__ px,
                                                      const int64_t* __restrict__ nu,
                                                      double* __restrict__ terms) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_x * g.n_x) return;
    double gt, eb;
    tab_cost(g, tab, consts[0], consts[1], make_pt2(g, i), nu[2 * i], nu[2 * i + 1], gt, eb);
    terms[i] = px[i] * gt;
}

// Normalised one-dimensional noise weights (the factors of phi2).
__global__ void k2_phin(G2 g, const double* __restrict__ p1, const double* __restrict__ sums,
                        double* __restrict__ phin) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.n_w) phin[c] = __ddiv_rn(p1[c], sums[1]);
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
    if (p.direct < 0 || p.direct > 3) return "direct must be in 0..3";
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
    g->direct = p.direct;
    g->tab_lo = -g->n_w - 1;
    g->tab_n = g->n_y + g->n_w + 2;
    g->ext_n = g->tab_n + g->n_w - 1;
    // Table cost against the exact fixed-order cost: below (2 n_w + 170) u M
    // by a forward error analysis (M the magnitude bound of the terms); taken
    // with a margin of two.
    g->eps_k = (double)(4 * g->n_w + 512) * 0x1p-53;
    // Double-float assembly of a table cost: about 60 operations, each within
    // 5 2^-48 of the magnitudes bounded by M, and the tables' own rounding to
    // pairs (2^-48): below 2^-39.5 M; taken as 2^-37 on top of eps_k.
    g->use_df = g->shift <= 24;
    g->eps_df = g->eps_k + 0x1p-37;
    g->eps_df_f = (float)g->eps_df * (1.0f + 0x1p-20f);   // rounded up
    {
        const double us = ldexp(p.delta, -g->shift);
        g->us_hi = (float)us;
        g->us_lo = (float)(us - (double)g->us_hi);
        g->inv_one_f = (float)ldexp(1.0, -g->shift);
        g->kk_hi = (float)g->kk;
        g->kk_lo = (float)(g->kk - (double)g->kk_hi);
    }
    // Source splits of the factorised u1 sums: about four blocks per SM.
    {
        const int64_t tiles = (g->n_y + 31) / 32, want = (4 * 152 + tiles * tiles - 1) /
                                                         (tiles * tiles);
        const int64_t n = g->n_x * g->n_x;
        g->u1_splits = (int32_t)(want < 1 ? 1 : (want > 64 ? 64 : (want > n ? n : want)));
    }
    const double vmax = (double)(g->hr + g->q + g->hx + g->hy + g->hw) * (double)g->one;
    if (!(vmax < 4.0e15)) return "lattice indices would overflow";
    return nullptr;
}

void launch2_setup(const G2& g, Dev2& d, int from_table, cudaStream_t s) {
    const int64_t n = g.n_x * g.n_x, big = n > g.n_w * g.n_w ? n : g.n_w * g.n_w;
    k2_exps<<<nblk(n > g.n_w ? n : g.n_w, 256), 256, 0, s>>>(g, d.px, d.phi1);
    k2_fixed_sum<<<1, 1024, 8 * sum_chunks(n), s>>>(d.px, n, 1.0, d.scratch);
    k2_fixed_sum<<<1, 1024, 8 * sum_chunks(g.n_w), s>>>(d.phi1, g.n_w, 1.0, d.scratch + 1);
    k2_scale_init<<<nblk(big, 256), 256, 0, s>>>(g, d.px, d.phi1, d.phi2, d.scratch, d.nu[0],
                                                 d.table, from_table);
    k2_phin<<<nblk(g.n_w, 256), 256, 0, s>>>(g, d.phi1, d.scratch, d.phin);
}

void launch2_sweep(const G2& g, Dev2& d, int cur, cudaStream_t s, Prof* prof) {
    ProfScope ps(prof, "search");
    const int64_t n = g.n_x * g.n_x;
    if (g.direct & 1) {
        k2_search<<<nblk(32 * n, kSearch2T), kSearch2T, 0, s>>>(g, d.phi2, d.U, d.nu[cur],
                                                                d.nu[cur ^ 1], d.idx);
        return;
    }
    k2_search_scr<<<nblk(32 * n, kSearch2T), kSearch2T, 0, s>>>(
        g, d.phi2, d.U, d.tab, d.tabf, d.scratch + 2, d.nu[cur], d.nu[cur ^ 1], d.idx);
}

void launch2_mmse(const G2& g, Dev2& d, int buf, cudaStream_t s, Prof* prof) {
    if (g.direct & 2) {
        ProfScope ps(prof, "u1_direct");
        k2_mmse<<<nblk(g.n_y * g.n_y, 128), 128, 0, s>>>(g, d.nu[buf], d.U);
        return;
    }
    const int64_t n = g.n_x * g.n_x, tiles = (g.n_y + kU1Tile - 1) / kU1Tile;
    const int64_t len = (n + g.u1_splits - 1) / g.u1_splits;
    float2* fa = reinterpret_cast<float2*>(d.fa);
    float2* fb = reinterpret_cast<float2*>(d.fb);
    {
        ProfScope ps(prof, "u1_shifts");
        k2_u1_sources<<<nblk(n, 256), 256, 0, s>>>(g, d.nu[buf], d.fv);
        k2_u1_mins<<<(unsigned)(2 * g.n_y), 256, 0, s>>>(g, d.fv, d.mins);
    }
    {
        ProfScope ps(prof, "u1_factors");
        k2_u1_factors<<<nblk(n * g.n_y, 256), 256, 0, s>>>(g, d.mins, d.fv, fa, fb, d.fa64,
                                                           d.fb64);
    }
    {
        ProfScope ps(prof, "u1_sums");
        k2_u1_sums<<<dim3((unsigned)tiles, (unsigned)tiles, (unsigned)g.u1_splits), 256, 0, s>>>(
            g, fa, fb, d.fv, len, d.part, reinterpret_cast<unsigned long long*>(d.scratch + 4));
    }
    {
        ProfScope ps(prof, "u1_finish");
        cudaMemsetAsync(d.list, 0, sizeof(int32_t), s);
        k2_u1_finish<<<nblk(g.n_y * g.n_y, 128), 128, 0, s>>>(g, d.part, g.u1_splits, d.U,
                                                             d.list);
        k2_u1_wide<<<(unsigned)(4 * 152), 128, 0, s>>>(g, d.nu[buf], d.fa64, d.fb64, d.fv,
                                                       d.list, d.U);
    }
}

void launch2_J(const G2& g, Dev2& d, int buf, double* out, cudaStream_t s, Prof* prof) {
    ProfScope ps(prof, "tables_J");
    const int64_t n = g.n_x * g.n_x;
    if (!(g.direct & 1)) {
        // The tables of the new u1 table: J's terms now, the next search later.
        cudaMemsetAsync(d.scratch + 2, 0, sizeof(double), s);
        k2_tab_consts<<<nblk(2 * g.n_y * g.n_y, 256), 256, 0, s>>>(g, d.U, d.phin, d.scratch + 2);
        k2_tab_rows<<<nblk(g.ext_n * g.tab_n, 256), 256, 0, s>>>(g, d.U, d.phin, d.H);
        k2_tab_cols<<<nblk(g.tab_n * g.tab_n, 256), 256, 0, s>>>(g, d.H, d.phin, d.tab, d.tabf);
        k2_J_terms_tab<<<nblk(n, 256), 256, 0, s>>>(g, d.tab, d.scratch + 2, d.px, d.nu[buf],
                                                    d.terms);
        k2_fixed_sum<<<1, 1024, 8 * sum_chunks(n), s>>>(d.terms, n, 0.5, out);
        return;
    }
    k2_J_terms<<<nblk(32 * n, kSearch2T), kSearch2T, 0, s>>>(g, d.phi2, d.U, d.px, d.nu[buf],
                                                             d.terms);
    k2_fixed_sum<<<1, 1024, 8 * sum_chunks(n), s>>>(d.terms, n, 0.5, out);
}

void launch2_table(const G2& g, Dev2& d, int buf, cudaStream_t s) {
    k2_table<<<nblk(2 * g.n_x * g.n_x, 256), 256, 0, s>>>(g, d.table, d.nu[buf]);
}

}  // namespace ucp
