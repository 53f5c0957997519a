// kernels_u1.cu -- the u1 step of the fast path (precision = 1):
//   U_j = E[x1 | y1 = y_j] = sum_i e^{-e_ij} f_i / sum_i e^{-e_ij},
//   e_ij = p_i + (y_j - f_i)^2 / 2,  p_i = x_i^2 / (2 sigma^2),
// the closed form of Section IV-C with x1 = f(x0) on the x0 grid and the
// Gaussian noise of Section V-A.
//
// Runs.  Targets are taken in runs of R (j0 = rR, ..., j0 + R - 1).  Within a
// run every weight of target j is scaled by the same factor
// exp(m_r + (y_j^2 - y_j0^2) / 2), which cancels in the ratio, leaving
//   w_ik = exp(m_r - e_{i,j0}) exp(k delta f_i)        (j = j0 + k),
// one exponential per (source, run) and one product per target.  m_r is a
// lower bound of min_i e_{i,j0}; it only sets the floating-point scale.
//
// Boxes.  Sources are cut into tiles of consecutive x0 points and each tile,
// greedily, into at most kBoxMax boxes of consecutive sources whose f values
// lie within 2 kHMax.  For a box with centre c, d_i = f_i - c (|d_i| <= h),
// a power of two s >= h, pm = min_i (p_i + d_i^2/2), q_i = exp(pm - p_i -
// d_i^2/2) and moments M_n = sum_i q_i (d_i / s)^n, the box's share of a
// target with z = y_j - c and u = z s is
//   sum_i w_ik     = A C^k sum_n u^n M_n / n!,
//   sum_i w_ik f_i = A C^k sum_n u^n (c M_n + s M_{n+1}) / n!,
//   A = exp(m_r - pm - (y_j0 - c)^2 / 2),  C = exp(delta c),
// the Taylor form of the fast Gauss transform (Greengard and Strain, SIAM J.
// Sci. Stat. Comput. 12, 1991).  With zeta = |z| h the tail after p terms is
// at most e^{2 zeta} zeta^p / p! of the box's exact share; p is chosen per
// (box, run) so that this is below 2^-52, and the expansion is used only
// where zeta <= kZetaMax and it is cheaper than the direct sum over the
// box's sources, which is taken otherwise.  Terms whose bound is below 2^-28
// are summed in FP32, the rest in double-float.
//
// Negligible work is skipped: a (box, run) or (source, run) pair is left out
// when every weight it holds is below e^-46 of its target's largest.
//
// Every sum runs in a fixed order (per run: the boxes of a tile in order;
// per target: the tiles in order), so results are bit-reproducible and the
// same alone or in a batch.
#include <float.h>

#include "df.cuh"
#include "ucp_fast.cuh"

namespace ucp {

namespace {

constexpr float kCut = 46.0f;       // skip weights below e^-46 of the maximum
constexpr float kHMax = 0.05f;      // box half width aimed at when grouping
constexpr float kHMoments = 0.25f;  // boxes wider than this get no moments
constexpr float kZetaMax = 1.0f;    // largest |y - c| h expanded
constexpr int kU1Runs = 32;         // runs per block of the u1 kernel (1 warp)
constexpr int kBuildT = 256;        // threads per tile of the single-instance box kernel
constexpr int kBuildTB = 512;       // threads per tile of the batched box kernel
constexpr int kBoxDF = 16;          // moments up to this order in double-float
constexpr unsigned kFull = 0xffffffffu;

// ---- sources and boxes ----------------------------------------------------------

// One block per tile (NW warps).
//  1. Every thread: per source f_i and exp(delta f_i) (double-float).
//  2. Warp 0: greedy grouping of consecutive sources into boxes whose f
//     values (leading floats) span at most 2 kHMax; the last box of a tile
//     takes whatever is left once kBoxMax - 1 boxes are closed.
//  3. One warp per box: centre c, half width h, scale pm, smallest prior.
//  4. The 32-source chunks of the boxes narrow enough to be expanded, spread
//     over the warps: every lane forms its source's terms q_i (d_i / s)^n,
//     n <= kBoxTerms, in shared memory, and lane n adds term n over the
//     chunk's sources in index order (the chunk's partial moment n).
//  5. One warp per expanded box: lane n adds the box's chunk partials in
//     chunk order (a fixed order), then the Taylor coefficients and exp(delta c).
struct BoxTerms {
    dfloat d[kBoxDF + 1];             // orders 0..kBoxDF in double-float
    float f[kBoxTerms - kBoxDF];      // the higher ones in FP32
};
constexpr int kChunkFast = 256;   // chunks whose f range the grouping reads at once
template <int NW>
struct BuildSmemT {
    int32_t s0[kBoxMax], n[kBoxMax];
    float fmin[kBoxMax], fmax[kBoxMax];
    float c[kBoxMax], pm[kBoxMax], sc[kBoxMax];
    int32_t ch0[kBoxMax + 1];          // first chunk of each box (expanded boxes)
    int32_t nch[kBoxMax];              // chunks of each box (0: not expanded)
    int nb;
    float cmin[kChunkFast], cmax[kChunkFast];   // f range of each 32-source chunk
    BoxTerms terms[NW][32];             // per warp, per lane (source)
};

template <int NW>
__device__ __forceinline__ void box_range(const FastView& f, BuildSmemT<NW>& sm, int64_t slot,
                                          int k, int lane) {
    const int64_t s0 = sm.s0[k];
    const int n = sm.n[k];
    const float c = 0.5f * (sm.fmin[k] + sm.fmax[k]);
    float hv = 0.0f, pv = FLT_MAX, pmn = FLT_MAX;
    for (int s = lane; s < n; s += 32) {
        const dfloat d = df_add_f(f.src_f[s0 + s], -c);
        const float pr = f.prior[s0 + s].hi;
        hv = fmaxf(hv, fabsf(d.hi) + fabsf(d.lo));
        pv = fminf(pv, fmaf(0.5f * d.hi, d.hi, pr));
        pmn = fminf(pmn, pr);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        hv = fmaxf(hv, __shfl_xor_sync(kFull, hv, o));
        pv = fminf(pv, __shfl_xor_sync(kFull, pv, o));
        pmn = fminf(pmn, __shfl_xor_sync(kFull, pmn, o));
    }
    const float h = hv * (1.0f + 0x1p-20f);
    const bool expand = h <= kHMoments;
    int e2 = 0;
    frexpf(h, &e2);                        // h < 2^e2
    const float sc = h > 0.0f ? ldexpf(1.0f, e2) : 1.0f;
    if (lane == 0) {
        f.box_geo[slot] = make_float4(c, h, pv, pmn);
        f.box_rng[slot] = make_float4(sm.fmin[k], sm.fmax[k], expand ? h : INFINITY, sc);
        sm.c[k] = c;
        sm.pm[k] = pv;
        sm.sc[k] = sc;
        sm.nch[k] = expand ? (n + 31) / 32 : 0;
    }
}

// Partial moments of sources b .. b + 31 of box k into part[0 .. kBoxTerms].
template <int NW>
__device__ __forceinline__ void chunk_moments(const FastView& f, BuildSmemT<NW>& sm, int k, int b,
                                              int warp, int lane, dfloat* part) {
    const int64_t s0 = sm.s0[k];
    const int cn = min(32, sm.n[k] - b);
    const float c = sm.c[k], pm = sm.pm[k];
    const float inv_sc = 1.0f / sm.sc[k];   // exact: a power of two
    BoxTerms* tw = sm.terms[warp];
    if (lane < cn) {
        const int64_t i = s0 + b + lane;
        const dfloat d = df_add_f(f.src_f[i], -c);
        dfloat ex = df_add_f(df_neg(f.prior[i]), pm);
        ex = df_add(ex, df_mul_f(df_mul(d, d), -0.5f));
        if (ex.hi < -87.0f) ex = {-87.0f, 0.0f};
        dfloat q = df_exp(ex, f.t64);
        const dfloat ds = {d.hi * inv_sc, d.lo * inv_sc};   // d / s, |d / s| <= 1
        BoxTerms& t = tw[lane];
#pragma unroll
        for (int m = 0; m <= kBoxDF; ++m) {
            t.d[m] = q;
            q = df_mul(q, ds);
        }
        float qf = q.hi;
#pragma unroll
        for (int m = 0; m < kBoxTerms - kBoxDF; ++m) {
            t.f[m] = qf;
            qf *= ds.hi;
        }
    }
    __syncwarp();
    if (lane <= kBoxDF) {
        dfloat M = {0.0f, 0.0f};
        for (int q = 0; q < cn; ++q) M = df_add(M, tw[q].d[lane]);
        part[lane] = M;
    } else if (lane <= kBoxTerms) {
        float a = 0.0f;
        for (int q = 0; q < cn; ++q) a += tw[q].f[lane - kBoxDF - 1];
        part[lane] = {a, 0.0f};
    }
    __syncwarp();
}

// Box k's moments from its chunk partials (in chunk order), Taylor
// coefficients and exp(delta c).
template <int NW>
__device__ __forceinline__ void box_coefs(const Geom& g, const FastView& f, BuildSmemT<NW>& sm,
                                          int64_t slot, int k, int lane,
                                          const dfloat* part) {
    const int q0 = sm.ch0[k], q1 = sm.ch0[k + 1];
    const float c = sm.c[k], sc = sm.sc[k];
    dfloat M = {0.0f, 0.0f};   // lane n <= kBoxTerms: moment n
    if (lane <= kBoxDF) {
        for (int q = q0; q < q1; ++q) M = df_add(M, part[(size_t)q * (kBoxTerms + 1) + lane]);
    } else if (lane <= kBoxTerms) {
        float a = 0.0f;
        for (int q = q0; q < q1; ++q) a += part[(size_t)q * (kBoxTerms + 1) + lane].hi;
        M = {a, 0.0f};
    }
    const dfloat M1 = {__shfl_down_sync(kFull, M.hi, 1), __shfl_down_sync(kFull, M.lo, 1)};
    if (lane < kBoxTerms) {
        const dfloat inv = f.t64[47 + lane];   // 1 / lane!
        dfloat* co = f.box_coef + slot * (2 * kBoxTerms);
        co[lane] = df_mul(M, inv);
        co[kBoxTerms + lane] = df_mul(df_add(df_mul_f(M, c), df_mul_f(M1, sc)), inv);
    }
    // exp(delta c), used only by expanded boxes, on a lane without a moment
    if (lane == 31) f.box_C[slot] = df_from_double(exp(g.delta * (double)c));
}

template <int NW>
__device__ __forceinline__ void box_build_body(const Geom& g, const FastView& f,
                                               const int64_t* __restrict__ nu,
                                               BuildSmemT<NW>& sm, int64_t t) {
    const int64_t t0 = t * f.tile;
    const int64_t t1 = min(t0 + f.tile, g.n_x);
    const dfloat dl = {f.delta_hi, f.delta_lo};
    const dfloat step = {f.step_hi, f.step_lo};
    // every warp takes whole 32-source chunks (blockDim is a multiple of 32)
    for (int64_t b0 = t0 + (threadIdx.x & ~31); b0 < t1; b0 += blockDim.x) {
        const int64_t i = b0 + (threadIdx.x & 31);
        float lo = FLT_MAX, hi = -FLT_MAX;
        if (i < t1) {
            // f_i = nu_i delta 2^-shift in double-float (the lattice index is exact)
            const dfloat fv = df_mul(df_from_i64(nu[i]), step);
            f.src_nu[i] = nu[i];
            f.src_f[i] = fv;
            // exp(delta f_i) in double-float (|delta f_i| stays below ~0.8)
            f.src_F[i] = df_exp(df_mul(fv, dl), f.t64);
            lo = hi = fv.hi;
        }
        // the chunk's f range (leading floats), for the grouping below
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(kFull, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, o));
        }
        const int64_t c = (b0 - t0) >> 5;
        if ((threadIdx.x & 31) == 0 && c < kChunkFast) {
            sm.cmin[c] = lo;
            sm.cmax[c] = hi;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t slot0 = t * kBoxMax;
    if (warp == 0) {
        const float wmax = 2.0f * kHMax;
        int nb = 0;
        int64_t sb = t0;
        float bmin = FLT_MAX, bmax = -FLT_MAX;
        for (int64_t base = t0; base < t1; base += 32) {
            // a chunk that fits whole in the open box (or once no box may
            // close) closes nothing: every prefix spans no more than the chunk
            const int64_t c = (base - t0) >> 5;
            if (c < kChunkFast) {
                const float lo = fminf(bmin, sm.cmin[c]), hi = fmaxf(bmax, sm.cmax[c]);
                if (nb == kBoxMax - 1 || hi - lo <= wmax) {
                    bmin = lo;
                    bmax = hi;
                    continue;
                }
            }
            const int64_t i = base + lane;
            const bool valid = i < t1;
            const float fi = valid ? f.src_f[i].hi : 0.0f;
            int from = 0;
            for (;;) {
                const bool part = valid && lane >= from;
                float vmin = part ? fi : FLT_MAX, vmax = part ? fi : -FLT_MAX;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const float a = __shfl_up_sync(kFull, vmin, d);
                    const float b = __shfl_up_sync(kFull, vmax, d);
                    if (lane >= d) {
                        vmin = fminf(vmin, a);
                        vmax = fmaxf(vmax, b);
                    }
                }
                const float rmin = fminf(bmin, vmin), rmax = fmaxf(bmax, vmax);
                const bool bad = part && nb < kBoxMax - 1 && rmax - rmin > wmax;
                const unsigned m = __ballot_sync(kFull, bad);
                if (m == 0) {
                    bmin = __shfl_sync(kFull, rmin, 31);
                    bmax = __shfl_sync(kFull, rmax, 31);
                    break;
                }
                const int l = __ffs(m) - 1;   // first source that does not fit
                const float cmin = __shfl_sync(kFull, rmin, l > 0 ? l - 1 : 0);
                const float cmax = __shfl_sync(kFull, rmax, l > 0 ? l - 1 : 0);
                if (lane == 0) {
                    sm.s0[nb] = (int32_t)sb;
                    sm.n[nb] = (int32_t)(base + l - sb);
                    sm.fmin[nb] = l > from ? cmin : bmin;
                    sm.fmax[nb] = l > from ? cmax : bmax;
                }
                ++nb;
                sb = base + l;
                bmin = FLT_MAX;
                bmax = -FLT_MAX;
                from = l;
            }
        }
        if (lane == 0) {
            sm.s0[nb] = (int32_t)sb;
            sm.n[nb] = (int32_t)(t1 - sb);
            sm.fmin[nb] = bmin;
            sm.fmax[nb] = bmax;
            sm.nb = nb + 1;
            f.box_cnt[t] = nb + 1;
        }
    }
    __syncthreads();
    const int nb = sm.nb;
    if (threadIdx.x < nb) {
        f.box_s0[slot0 + threadIdx.x] = sm.s0[threadIdx.x];
        f.box_n[slot0 + threadIdx.x] = sm.n[threadIdx.x];
    }
    constexpr int kWarps = NW;
    for (int k = warp; k < nb; k += kWarps) box_range(f, sm, slot0 + k, k, lane);
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0;
        for (int k = 0; k < nb; ++k) {
            sm.ch0[k] = a;
            a += sm.nch[k];
        }
        sm.ch0[nb] = a;   // <= tile / 32 + nb <= box_cap
    }
    __syncthreads();
    const int total = sm.ch0[nb];
    dfloat* part = f.box_part + (size_t)t * (size_t)f.box_cap * (kBoxTerms + 1);
    for (int q = warp; q < total; q += kWarps) {
        int k = 0;
        while (sm.ch0[k + 1] <= q) ++k;   // the box of chunk q (the same for the warp)
        chunk_moments(f, sm, k, (q - sm.ch0[k]) * 32, warp, lane,
                      part + (size_t)q * (kBoxTerms + 1));
    }
    __syncthreads();
    for (int k = warp; k < nb; k += kWarps)
        if (sm.nch[k]) box_coefs(g, f, sm, slot0 + k, k, lane, part);
}

// ---- per-run scale and cut --------------------------------------------------

// One warp per run, from the box summaries:
//   run_lo <= min_i e_{i,j0}          (lower bound; the run's scale m_r)
//   run_hi >= min_i e_ij for every j of the run (upper bound; the cut).
// Over a box, e_i(y) >= pmin + dist(y, [fmin, fmax])^2 / 2 and
// e_i(y) >= pm + z^2/2 - h|z|; the source attaining pm has
// e(y) <= pm + z^2/2 + h|z| (z = y - c), convex in y.
constexpr int kRunT = 256;

// The instance's boxes, compacted in tile order, are spread over the lanes:
// each warp forms the prefix of the tiles' box counts (a shuffle scan; at
// most 32 tiles) and finds the tile of its box s by a binary search over the
// lanes.  The bounds are minima, so their order does not matter.
__device__ __forceinline__ void run_shift_body(const Geom& g, const FastView& f,
                                               int64_t bx) {
    const int lane = threadIdx.x & 31;
    const int64_t r = bx * (kRunT / 32) + (threadIdx.x >> 5);
    if (r >= f.n_runs) return;   // the same for the warp
    int end = lane < f.n_tiles ? f.box_cnt[lane] : 0;   // boxes of tiles 0..lane
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(kFull, end, d);
        if (lane >= d) end += o;
    }
    const int nbox = __shfl_sync(kFull, end, 31);
    const int64_t j0 = r * f.run;
    const float ya = (float)((double)(j0 - g.hy) * g.delta);
    const float yb = (float)((double)(j0 + f.run - 1 - g.hy) * g.delta);
    float lo = FLT_MAX, hi = FLT_MAX;
    for (int b0 = 0; b0 < nbox; b0 += 32) {
        const int s = b0 + lane;
        // first tile whose running count exceeds s
        int t = 0;
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) {
            const int e = __shfl_sync(kFull, end, t + w - 1);
            if (e <= s) t += w;
        }
        const int prev = __shfl_sync(kFull, end, t > 0 ? t - 1 : 0);   // boxes before tile t
        if (s >= nbox) continue;
        const int64_t slot = (int64_t)t * kBoxMax + (s - (t > 0 ? prev : 0));
        const float4 geo = f.box_geo[slot];
        const float4 rg = f.box_rng[slot];
        const float d1 = fmaxf(0.0f, fmaxf(rg.x - ya, ya - rg.y));
        const float lb1 = fmaf(0.5f * d1, d1, geo.w);
        const float za = fabsf(ya - geo.x);
        const float lb2 = za >= geo.y ? geo.z + za * (0.5f * za - geo.y)
                                      : geo.z - 0.5f * geo.y * geo.y;
        lo = fminf(lo, fmaxf(lb1, lb2));
        const float zm = fmaxf(za, fabsf(yb - geo.x));
        hi = fminf(hi, geo.z + zm * (0.5f * zm + geo.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(kFull, lo, o));
        hi = fminf(hi, __shfl_xor_sync(kFull, hi, o));
    }
    if (lane == 0) {
        f.run_lo[r] = lo - (0.01f + 1e-5f * fabsf(lo));
        f.run_hi[r] = hi + (0.01f + 1e-5f * fabsf(hi));
    }
}

// ---- the u1 sums ------------------------------------------------------------

// Taylor terms for zeta = |z| h: p = terms kept (tail bound <= 2^-52 of the
// box's share; -1 if more than kBoxTerms would be needed), n1 = first term
// summed in FP32 (its tail bound <= 2^-28, so the FP32 rounding of the tail
// is ~2^-52 of the share, below the double-float Horner steps' own).
// 1 / (n + 1) from a table (the factor 1.001 on zeta covers its rounding).
__constant__ float kInvN[kBoxTerms + 1] = {
    1.0f / 1, 1.0f / 2, 1.0f / 3, 1.0f / 4, 1.0f / 5, 1.0f / 6, 1.0f / 7, 1.0f / 8, 1.0f / 9,
    1.0f / 10, 1.0f / 11, 1.0f / 12, 1.0f / 13, 1.0f / 14, 1.0f / 15, 1.0f / 16, 1.0f / 17,
    1.0f / 18, 1.0f / 19, 1.0f / 20, 1.0f / 21, 1.0f / 22, 1.0f / 23, 1.0f / 24, 1.0f / 25};
static_assert(kBoxTerms == 24, "reciprocal table length");
__device__ __forceinline__ void taylor_terms(float zeta, int& n1, int& p) {
    float term = expf(2.0f * zeta) * 1.001f;   // e^{2 zeta} zeta^n / n!, n = 0
    const float zs = zeta * 1.001f;
    n1 = -1;
    p = -1;
    for (int n = 0; n <= kBoxTerms; ++n) {
        if (n1 < 0 && term <= 0x1p-28f) n1 = n;
        if (term <= 0x1p-52f) {
            p = n;
            break;
        }
        term *= zs * kInvN[n];
    }
    if (n1 < 0) n1 = p;
}

// Box share by its Taylor expansion, added to the sums of targets
// kq0 .. kq0 + TR - 1 of the run (R targets).  z and the factor E C^k of
// target k are advanced from target 0 one step at a time, so every target
// gets the same operations whichever thread evaluates it.
template <int R, int TR>
__device__ __forceinline__ void fgt_box(const FastView& f, int64_t slot, float c,
                                        float pm, float sc, dfloat y0, dfloat dl,
                                        float m_lo, int p, int n1, const dfloat* st64,
                                        int kq0, dfloat (&N)[TR], dfloat (&D)[TR]) {
    const dfloat* __restrict__ ca = f.box_coef + slot * (2 * kBoxTerms);
    const dfloat* __restrict__ cb = ca + kBoxTerms;
    const dfloat z0 = df_add_f(y0, -c);
    float sh, sl;
    two_sum(m_lo, -pm, sh, sl);
    dfloat ex = df_add(df_norm(sh, sl), df_mul_f(df_mul(z0, z0), -0.5f));
    if (ex.hi < -87.0f) ex = {-87.0f, 0.0f};
    dfloat E = df_exp(ex, st64);
    const dfloat C = f.box_C[slot];
    // u = z s and its step delta s (scaling by a power of two is exact)
    dfloat z = {z0.hi * sc, z0.lo * sc};
    const dfloat du = {dl.hi * sc, dl.lo * sc};
    for (int k = 0; k < kq0; ++k) {
        z = df_add(z, du);
        E = df_mul(E, C);
    }
    constexpr int Q = TR < 4 ? TR : 4;
#pragma unroll
    for (int k0 = 0; k0 < TR; k0 += Q) {
        dfloat zq[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            zq[q] = z;
            z = df_add(z, du);
        }
        float tD[Q], tN[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) tD[q] = tN[q] = 0.0f;
        for (int n = p - 1; n >= n1; --n) {
            const float an = ca[n].hi, bn = cb[n].hi;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                tD[q] = fmaf(tD[q], zq[q].hi, an);
                tN[q] = fmaf(tN[q], zq[q].hi, bn);
            }
        }
        dfloat aD[Q], aN[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            aD[q] = {tD[q], 0.0f};
            aN[q] = {tN[q], 0.0f};
        }
        for (int n = n1 - 1; n >= 0; --n) {
            const dfloat an = ca[n], bn = cb[n];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                aD[q] = df_add(df_mul(aD[q], zq[q]), an);
                aN[q] = df_add(df_mul(aN[q], zq[q]), bn);
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            D[k0 + q] = df_add(D[k0 + q], df_mul(E, aD[q]));
            N[k0 + q] = df_add(N[k0 + q], df_mul(E, aN[q]));
            if (kq0 + k0 + q + 1 < R) E = df_mul(E, C);
        }
    }
}

// Box share by the direct sum over its sources (two recurrences at a time),
// skipping sources whose weights are all negligible, for targets kq0 .. kq0 +
// TR - 1 of the run (the weight advanced from target 0 one step at a time).
// Returns the number of (source, run) pairs evaluated.
template <int R, int TR>
__device__ __forceinline__ unsigned direct_box(const FastView& f, int64_t s0, int n,
                                               float ya, float yb, float cut,
                                               float m_lo, int64_t ybase,
                                               const dfloat* st64, int kq0,
                                               dfloat (&N)[TR], dfloat (&D)[TR]) {
    const dfloat step = {f.step_hi, f.step_lo};
    unsigned evaluated = 0;
    int s = 0;
    while (s < n) {
        int64_t sel0 = 0, sel1 = 0;
        int ns = 0;
        for (; s < n && ns < 2; ++s) {
            const int64_t i = s0 + s;
            const float fh = f.src_f[i].hi;
            const float dmin = fmaxf(0.0f, fmaxf(ya - fh, fh - yb));
            if (fmaf(0.5f * dmin, dmin, f.prior[i].hi) <= cut) {
                if (ns == 0) sel0 = i;
                else sel1 = i;
                ++ns;
            }
        }
        if (ns == 0) break;
        if (ns == 1) sel1 = sel0;
        evaluated += (unsigned)ns;
        dfloat w[2], F[2], fv[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int64_t i = q == 0 ? sel0 : sel1;
            fv[q] = f.src_f[i];
            F[q] = f.src_F[i];
            // w = exp(m_r - p_i - (y_j0 - f_i)^2 / 2), y_j0 - f_i exact in units of step
            const dfloat d0 = df_mul(df_from_i64(ybase - f.src_nu[i]), step);
            dfloat ex = df_add(f.prior[i], df_mul_f(df_mul(d0, d0), 0.5f));
            ex = df_add_f(df_neg(ex), m_lo);
            if (ex.hi < -87.0f) ex = {-87.0f, 0.0f};
            w[q] = df_exp(ex, st64);
        }
        if (ns == 1) w[1] = {0.0f, 0.0f};
        for (int k = 0; k < kq0; ++k) {
            w[0] = df_mul(w[0], F[0]);
            w[1] = df_mul(w[1], F[1]);
        }
#pragma unroll
        for (int k = 0; k < TR; ++k) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float pp, pe;
                df_mul_raw(w[q], fv[q], pp, pe);
                N[k] = df_acc(N[k], pp, pe);
                D[k] = df_add(D[k], w[q]);
                if (kq0 + k + 1 < R) w[q] = df_mul(w[q], F[q]);
            }
        }
    }
    return evaluated;
}

// Threads per run of R targets when a launch is small: P = 4 (each takes R / 4
// consecutive targets and repeats the run's exponentials), so that a single
// instance's few runs fill more of the GPU; launches that fill it anyway run
// one thread per run (P = 1).  Every target gets the same operations either
// way.
template <int R>
constexpr int u1_parts() { return R >= 4 ? 4 : 1; }
constexpr int64_t kU1SplitMaxBlocks = 4 * 152;   // launches up to this many blocks split

// Block (bx, t): runs bx*kU1Runs.. against the boxes of tile t, thread
// (part, run) taking targets part * TR .. + TR - 1 of its run (TR = R / P);
// writes the tile's partial sums of those targets.
template <int R, int P>
__device__ __forceinline__ void u1_main_body(const Geom& g, const FastView& f,
                                             dfloat* st64, int64_t bx, int64_t t) {
    constexpr int TR = R / P;
    for (int k = threadIdx.x; k < 47; k += blockDim.x) st64[k] = f.t64[k];
    __syncthreads();
    const int part = threadIdx.x / kU1Runs;
    const int kq0 = part * TR;
    const int64_t r0 = bx * kU1Runs + threadIdx.x % kU1Runs;
    const int64_t r = r0 < f.n_runs ? r0 : f.n_runs - 1;
    const int64_t j0 = r * R;
    const float m_lo = f.run_lo[r];
    const float cut = kCut + f.run_hi[r] + 0.01f;
    const float ya = (float)((double)(j0 - g.hy) * g.delta);
    const float yb = (float)((double)(j0 + R - 1 - g.hy) * g.delta);
    const dfloat dl = {f.delta_hi, f.delta_lo};
    const dfloat y0 = df_mul(df_from_i64(j0 - g.hy), dl);
    const int64_t ybase = (j0 - g.hy) * g.one;
    dfloat N[TR], D[TR];
#pragma unroll
    for (int k = 0; k < TR; ++k) N[k] = D[k] = {0.0f, 0.0f};
    unsigned n_dir = 0, n_box = 0, t_df = 0, t_f32 = 0;
    const int nb = f.box_cnt[t];
    for (int k = 0; k < nb; ++k) {
        const int64_t slot = t * kBoxMax + k;
        const float4 geo = f.box_geo[slot];   // c, h, pm, pmin
        const float4 rg = f.box_rng[slot];    // fmin, fmax, h (expandable) or inf
        // lower bound of e over (box, run); skip the box if it exceeds the cut
        const float d1 = fmaxf(0.0f, fmaxf(rg.x - yb, ya - rg.y));
        const float lb1 = fmaf(0.5f * d1, d1, geo.w);
        const float dz = fmaxf(0.0f, fmaxf(geo.x - yb, ya - geo.x));
        const float lb2 = dz >= geo.y ? geo.z + dz * (0.5f * dz - geo.y)
                                      : geo.z - 0.5f * geo.y * geo.y;
        const float lb = fmaxf(lb1, lb2);
        if (lb - 1e-5f * (1.0f + fabsf(lb)) > cut) continue;
        const int n = f.box_n[slot];
        const float zeta = rg.z * fmaxf(fabsf(ya - geo.x), fabsf(yb - geo.x)) * 1.001f;
        int p = -1, n1 = 0;
        if (zeta <= kZetaMax) {
            taylor_terms(zeta, n1, p);
            if (p >= 0) {
                const int cf = R * (2 * (18 * n1 + 2 * (p - n1)) + 40) + 300;
                const int cd = n * (30 * R + 130);
                if (cf >= cd) p = -1;
            }
        }
        if (p >= 0) {
            fgt_box<R, TR>(f, slot, geo.x, geo.z, rg.w, y0, dl, m_lo, p, n1, st64, kq0, N, D);
            ++n_box;
            t_df += (unsigned)n1;
            t_f32 += (unsigned)(p - n1);
        } else {
            n_dir += direct_box<R, TR>(f, f.box_s0[slot], n, ya, yb, cut, m_lo, ybase,
                                       st64, kq0, N, D);
        }
    }
    if (r0 >= f.n_runs) return;
    if (f.n_pairs && part == 0) {
        if (n_dir) atomicAdd((unsigned long long*)f.n_pairs, (unsigned long long)n_dir);
        if (n_box) {
            atomicAdd((unsigned long long*)f.n_pairs + 1, (unsigned long long)n_box);
            atomicAdd((unsigned long long*)f.n_pairs + 2, (unsigned long long)t_df * (2 * R));
            atomicAdd((unsigned long long*)f.n_pairs + 3, (unsigned long long)t_f32 * (2 * R));
        }
    }
    dfloat* pN = f.partN + (size_t)t * g.n_y;
    dfloat* pD = f.partD + (size_t)t * g.n_y;
#pragma unroll
    for (int k = 0; k < TR; ++k)
        if (j0 + kq0 + k < g.n_y) {
            pN[j0 + kq0 + k] = N[k];
            pD[j0 + kq0 + k] = D[k];
        }
}

// U_j = sum over tiles of the numerator partials / of the denominator
// partials.  The double-float partials are added with accurate additions
// (error <= 3 u^2 of each result) in a fixed tree; the ratio in FP64.
__device__ __forceinline__ void u1_combine_body(const Geom& g, const FastView& f,
                                                double* __restrict__ U, int64_t bx) {
    const int64_t j = bx * blockDim.x + threadIdx.x;
    if (j >= g.n_y) return;
    // tiles in groups of 8: each group summed as a pairwise tree, the group
    // sums added in order (a fixed order, depth 3 + groups)
    dfloat n = {0.0f, 0.0f}, d = {0.0f, 0.0f};
    for (int t0 = 0; t0 < f.n_tiles; t0 += 8) {
        dfloat pn[8], pd[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {   // issue the loads, then sum
            const bool in = t0 + k < f.n_tiles;
            const int t = in ? t0 + k : t0;
            pn[k] = in ? f.partN[(size_t)t * g.n_y + j] : dfloat{0.0f, 0.0f};
            pd[k] = in ? f.partD[(size_t)t * g.n_y + j] : dfloat{0.0f, 0.0f};
        }
#pragma unroll
        for (int w = 1; w < 8; w <<= 1)
#pragma unroll
            for (int k = 0; k < 8; k += 2 * w) {
                pn[k] = df_add_acc(pn[k], pn[k + w]);
                pd[k] = df_add_acc(pd[k], pd[k + w]);
            }
        n = df_add_acc(n, pn[0]);
        d = df_add_acc(d, pd[0]);
    }
    U[j] = df_to_double(n) / df_to_double(d);
}

// ---- single-instance kernels --------------------------------------------------

__global__ void __launch_bounds__(kBuildT) k_box_build(Geom g, FastView f,
                                                      const int64_t* __restrict__ nu) {
    __shared__ BuildSmemT<kBuildT / 32> sm;
    box_build_body<kBuildT / 32>(g, f, nu, sm, blockIdx.x);
}

__global__ void __launch_bounds__(kRunT) k_run_shift(Geom g, FastView f) {
    run_shift_body(g, f, blockIdx.x);
}

template <int R, int P>
__global__ void __launch_bounds__(kU1Runs * P) k_u1_main(Geom g, FastView f) {
    __shared__ dfloat st64[47];
    u1_main_body<R, P>(g, f, st64, blockIdx.x, blockIdx.y);
}

__global__ void k_u1_combine(Geom g, FastView f, double* __restrict__ U) {
    u1_combine_body(g, f, U, blockIdx.x);
}

// ---- batched wrappers -----------------------------------------------------------
// The block map gives (instance, block of that instance's own grid); the
// instance descriptor is staged in shared memory and the body runs unchanged.

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

// NW warps per tile, the per-warp term scratch in dynamic shared memory.  A
// launch of few tiles (a single instance) takes twice the warps of the
// single-instance kernel, spreading a tile's boxes and chunks wider; each
// chunk's and box's sums are the same either way.
template <int NW>
__global__ void __launch_bounds__(NW * 32) kb_box_build(const InstDev* insts,
                                                       const BlockRef* map) {
    __shared__ InstDev sd;
    extern __shared__ __align__(16) char box_smem[];
    BuildSmemT<NW>& sm = *reinterpret_cast<BuildSmemT<NW>*>(box_smem);
    const BlockRef r = stage(insts, map, sd);
    box_build_body<NW>(sd.g, sd.f, sd.nu[sd.cur ^ 1], sm, r.local);
}

__global__ void __launch_bounds__(kRunT) kb_run_shift(const InstDev* insts,
                                                      const BlockRef* map) {
    __shared__ InstDev sd;
    const BlockRef r = stage(insts, map, sd);
    run_shift_body(sd.g, sd.f, r.local);
}

template <int R, int P>
__global__ void __launch_bounds__(kU1Runs * P) kb_u1_main(const InstDev* insts,
                                                          const BlockRef* map) {
    __shared__ InstDev sd;
    __shared__ dfloat st64[47];
    const BlockRef r = stage(insts, map, sd);
    const int64_t rb = sd.f.r_blocks;
    u1_main_body<R, P>(sd.g, sd.f, st64, r.local % rb, r.local / rb);
}

// Batched launches split runs of 16 targets whatever their size: one thread
// per 16-target run needs 168 registers and a large unrolled body (measured
// on 256 uneven instances: 34.1 ms against 39.7 ms per ten sweeps).
// P threads per run (0: the rule above).  Every target gets the same
// operations whichever P, so the results do not depend on it.
template <int R>
void launch_kb_u1_main(unsigned nb, const InstDev* d, const BlockRef* m, cudaStream_t s,
                       int P) {
    if (P == 0) P = (nb <= kU1SplitMaxBlocks || R == 16) ? u1_parts<R>() : 1;
    if (P >= 4 && R >= 4) {
        kb_u1_main<R, (R >= 4 ? 4 : 1)><<<nb, kU1Runs * 4, 0, s>>>(d, m);
    } else if (P >= 2 && R >= 2) {
        kb_u1_main<R, (R >= 2 ? 2 : 1)><<<nb, kU1Runs * 2, 0, s>>>(d, m);
    } else {
        kb_u1_main<R, 1><<<nb, kU1Runs, 0, s>>>(d, m);
    }
}

template <int R>
void launch_k_u1_main(dim3 grid, const Geom& g, const FastView& f, cudaStream_t s) {
    if ((int64_t)grid.x * grid.y <= kU1SplitMaxBlocks)
        k_u1_main<R, u1_parts<R>()><<<grid, kU1Runs * u1_parts<R>(), 0, s>>>(g, f);
    else
        k_u1_main<R, 1><<<grid, kU1Runs, 0, s>>>(g, f);
}

__global__ void kb_u1_combine(const InstDev* insts, const BlockRef* map) {
    __shared__ InstDev sd;
    const BlockRef r = stage(insts, map, sd);
    u1_combine_body(sd.g, sd.f, sd.U, r.local);
}

inline unsigned blocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// ---- host side ------------------------------------------------------------------

int mmse_run_length(const Geom& g) {
    // keep the exponent change along a run below ~15 (float range of the
    // double-float weights): R * delta * (Y + max |f|) <= 15
    const double F = (double)((g.hr + 2 * g.q) > g.hx ? (g.hr + 2 * g.q) : g.hx) * g.delta;
    const double slope = g.delta * ((double)g.hy * g.delta + F);
    int R = 16;
    while (R > 1 && (R - 1) * slope > 15.0) R /= 2;
    return R;
}

void u1_plan(const Geom& g, int max_tiles, FastPlan* fp) {
    fp->run = mmse_run_length(g);
    fp->n_runs = (g.n_y + fp->run - 1) / fp->run;
    fp->r_blocks = (fp->n_runs + kU1Runs - 1) / kU1Runs;
    int64_t tile = (g.n_x + max_tiles - 1) / max_tiles;
    tile = (tile + 31) / 32 * 32;
    if (tile < g.u1_tile_min) tile = g.u1_tile_min;
    fp->tile = tile;
    fp->n_tiles = (int)((g.n_x + tile - 1) / tile);
    fp->box_cap = (tile + 31) / 32 + kBoxMax;
}

size_t u1_scratch_bytes(const Geom& g, const FastPlan& fp, size_t align) {
    auto rnd = [align](size_t n) { return (n + align - 1) / align * align; };
    const size_t slots = (size_t)fp.n_tiles * kBoxMax;
    return 3 * rnd(8 * (size_t)g.n_x) +                       // src_nu, src_f, src_F
           rnd(4 * (size_t)fp.n_tiles) + 2 * rnd(4 * slots) +   // box_cnt, box_s0, box_n
           2 * rnd(16 * slots) + rnd(8 * slots) +                // box_geo, box_rng, box_C
           rnd(8 * slots * 2 * kBoxTerms) +                      // box_coef
           rnd(8 * (size_t)fp.n_tiles * (size_t)fp.box_cap * (kBoxTerms + 1)) +  // box_part
           2 * rnd(4 * (size_t)fp.n_runs) +                      // run_lo, run_hi
           2 * rnd(8 * (size_t)fp.n_tiles * (size_t)g.n_y);     // partN, partD
}

bool u1_carve(const Geom& g, FastView* f, void* (*get)(void*, size_t), void* ctx) {
    const size_t slots = (size_t)f->n_tiles * kBoxMax;
    f->src_nu = (int64_t*)get(ctx, 8 * (size_t)g.n_x);
    f->src_f = (dfloat*)get(ctx, 8 * (size_t)g.n_x);
    f->src_F = (dfloat*)get(ctx, 8 * (size_t)g.n_x);
    f->box_cnt = (int32_t*)get(ctx, 4 * (size_t)f->n_tiles);
    f->box_s0 = (int32_t*)get(ctx, 4 * slots);
    f->box_n = (int32_t*)get(ctx, 4 * slots);
    f->box_geo = (float4*)get(ctx, 16 * slots);
    f->box_rng = (float4*)get(ctx, 16 * slots);
    f->box_C = (dfloat*)get(ctx, 8 * slots);
    f->box_coef = (dfloat*)get(ctx, 8 * slots * 2 * kBoxTerms);
    f->box_part = (dfloat*)get(ctx, 8 * (size_t)f->n_tiles * (size_t)f->box_cap *
                                        (kBoxTerms + 1));
    f->run_lo = (float*)get(ctx, 4 * (size_t)f->n_runs);
    f->run_hi = (float*)get(ctx, 4 * (size_t)f->n_runs);
    f->partN = (dfloat*)get(ctx, 8 * (size_t)f->n_tiles * (size_t)g.n_y);
    f->partD = (dfloat*)get(ctx, 8 * (size_t)f->n_tiles * (size_t)g.n_y);
    return f->src_nu && f->src_f && f->src_F && f->box_cnt && f->box_s0 && f->box_n &&
           f->box_geo && f->box_rng && f->box_C && f->box_coef && f->box_part && f->run_lo &&
           f->run_hi && f->partN && f->partD;
}

void launch_mmse_fast(const Geom& g, const FastView& f, const int64_t* nu,
                      double* U, cudaStream_t s, Prof* prof) {
    cudaEvent_t ev;
    int k = prof ? prof->begin("u1_boxes", &ev) : -1;
    k_box_build<<<(unsigned)f.n_tiles, kBuildT, 0, s>>>(g, f, nu);
    if (prof) prof->end(k, ev);
    k = prof ? prof->begin("u1_shift", &ev) : -1;
    k_run_shift<<<blocks(f.n_runs, kRunT / 32), kRunT, 0, s>>>(g, f);
    if (prof) prof->end(k, ev);
    k = prof ? prof->begin("mmse_main", &ev) : -1;
    dim3 grid((unsigned)f.r_blocks, (unsigned)f.n_tiles);
    switch (f.run) {
        case 16: launch_k_u1_main<16>(grid, g, f, s); break;
        case 8: launch_k_u1_main<8>(grid, g, f, s); break;
        case 4: launch_k_u1_main<4>(grid, g, f, s); break;
        case 2: launch_k_u1_main<2>(grid, g, f, s); break;
        default: launch_k_u1_main<1>(grid, g, f, s); break;
    }
    if (prof) prof->end(k, ev);
    k = prof ? prof->begin("mmse_combine", &ev) : -1;
    k_u1_combine<<<blocks(g.n_y, 256), 256, 0, s>>>(g, f, U);
    if (prof) prof->end(k, ev);
}

cudaError_t u1_init_attributes() {
    const cudaError_t e = cudaFuncSetAttribute(kb_box_build<kBuildTB / 32>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sizeof(BuildSmemT<kBuildTB / 32>));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kb_box_build<kBuildT / 32>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(BuildSmemT<kBuildT / 32>));
}

int64_t u1_batch_blocks(const Geom& g, const FastPlan& fp, int kind) {
    switch (kind) {
        case kBTile: return fp.n_tiles;
        case kBRun: return (fp.n_runs + kRunT / 32 - 1) / (kRunT / 32);
    }
    (void)g;
    return 0;
}

int64_t batch_mmse_blocks(const Geom&, const FastPlan& fp) {
    return fp.r_blocks * fp.n_tiles;
}

void launch_batch_u1(const BatchLaunch& bl, cudaStream_t s, Prof* prof) {
    const InstDev* d = bl.insts;
    {
        ProfScope ps(prof, "u1_boxes");
        const unsigned nb = (unsigned)bl.n_blocks[kBTile];
        if (nb <= 2 * (unsigned)sm_count())
            kb_box_build<kBuildTB / 32><<<nb, kBuildTB, sizeof(BuildSmemT<kBuildTB / 32>), s>>>(
                d, bl.map[kBTile]);
        else
            kb_box_build<kBuildT / 32><<<nb, kBuildT, sizeof(BuildSmemT<kBuildT / 32>), s>>>(
                d, bl.map[kBTile]);
    }
    {
        ProfScope ps(prof, "u1_shift");
        kb_run_shift<<<(unsigned)bl.n_blocks[kBRun], kRunT, 0, s>>>(d, bl.map[kBRun]);
    }
    {
        ProfScope ps(prof, "mmse_main");
        for (int r = 0; r < 5; ++r) {
            if (bl.mmse_blocks[r] == 0) continue;
            const unsigned nb = (unsigned)bl.mmse_blocks[r];
            const BlockRef* m = bl.mmse_map[r];
            const int P = bl.u1_threads[r];
            switch (r) {
                case 0: launch_kb_u1_main<1>(nb, d, m, s, P); break;
                case 1: launch_kb_u1_main<2>(nb, d, m, s, P); break;
                case 2: launch_kb_u1_main<4>(nb, d, m, s, P); break;
                case 3: launch_kb_u1_main<8>(nb, d, m, s, P); break;
                default: launch_kb_u1_main<16>(nb, d, m, s, P); break;
            }
        }
    }
    ProfScope ps(prof, "mmse_combine");
    kb_u1_combine<<<(unsigned)bl.n_blocks[kBPerY], 256, 0, s>>>(d, bl.map[kBPerY]);
}

}  // namespace ucp
