// kernels_tc.cu -- the correlation tables of the fast path on the tensor
// cores (tcgen05, sm_103a).
//
// The u0 search evaluates S(u) through three correlations of the fixed
// Gaussian weights against E = U^(y) - y (kernels_fast.cu):
//   P_p = sum_l a_l E_{p+l} (a_l = phi_l w_l),  Q_p = sum_l phi_l E_{p+l}^2,
//   R_p = sum_l phi_l E_{p+l} E_{p+l+1}.
// Each is a Toeplitz product.  With p = 128 a + b and m = b + l,
//   y_{128a+b} = sum_m h_{m-b} x_{128a+m},
// i.e. D[b][a] = sum_m H[b][m] X[m][a]: a 128-row Toeplitz matrix of the
// filter times a Hankel matrix of the signal -- a GEMM with M = 128 phases,
// N = table columns (128 positions each), K = taps.
//
// Exactness (an Ozaki-style split).  The screening needs the tables to
// ~2^-40 of the cost, far beyond bf16.  The taps are cut into chunks of 128;
// per chunk the filter is scaled by a power of two sigma_h(c) >= its largest
// |h|, per 128-value block beta of the signal by sigma_x(beta) >= its largest
// |x|, and each scaled value v (|v| < 1) is cut into six 8-bit integer
// slices, v = sum_t s_t 2^-8(t+1) + r with |s_0| <= 256, |s_t| <= 128 and
// |r| <= 2^-49.  Integers up to 256 in magnitude are exact in bf16 and a
// product of two is exact in FP32.  Products (s, t) with s + t = k share
// accumulator k (k = 0..5, 21 products; s + t >= 6 is dropped); over 128 taps
// accumulator k sums at most 2 products bounded by 2^15 and k - 1 bounded by
// 2^14 (2^16 alone for k = 0): |sum| <= 2^23 + (k - 1) 2^21 <= 2^24, so the
// tensor core's FP32 accumulation is exact.  The six exact accumulators are
// folded in double-float and scaled.  Chunks are added
// in a fixed tree of accurate double-float additions.  Every rounding and
// truncation is bounded (tc_combine_body), and the bound per table column
// replaces the table term of the screening bound.
#include <cudaTypedefs.h>
#include <float.h>

#include <atomic>

#include "df.cuh"
#include "tc.cuh"
#include "ucp_fast.cuh"

namespace ucp {

namespace {

constexpr int kSl = kTcSlices;        // slices per operand
constexpr int kTcT = 512;             // threads of the tensor-core kernel
constexpr uint32_t kTcATile = 128 * 128 * 2;   // filter tile: 128 phases x 128 taps
constexpr uint32_t kTcBTile = 64 * 128 * 2;    // signal tile: 64 columns x 128 taps
constexpr uint32_t kTcHBytes = kSl * 8 * 256 * 2;   // a chunk's filter slices
constexpr int kTcABuf = 3;   // filter tiles in the ring, built ahead of the MMAs that read them
constexpr size_t kTcSmem = kSl * kTcBTile + kTcABuf * kTcATile + kTcHBytes + 1024;
constexpr uint32_t kTmemCols = 512;   // accumulator k at columns 64 k .. 64 k + 63 (k < 6)
constexpr int64_t kTcPolls = 4000000; // bound of every mbarrier wait
// Bound of the one wait the test hook (tc_err[1] != 0) leaves without its
// producer, which guards nothing in flight and may end early: hook 1 issues
// no filter-slice copy (the wait for it); hook 2 builds only the first filter
// tile (the MMA thread's wait for the second, after the first slice group is
// in flight; tc_hook_one_group).
constexpr int64_t kTcHookPolls = 20000;

__device__ __forceinline__ uint16_t bf16_bits(float v) {   // exact for |v| <= 256 integers
    return (uint16_t)(__float_as_uint(v) >> 16);
}

// ---- filter slices (once per instance) ------------------------------------

// Block b < 2 tc_nch: chunk c = b mod tc_nch of filter flt = b / tc_nch
// (0: a_l = phi_l w_l, 1: phi_l): window G[i] = h[128 c - 127 + i], i < 256,
// cut into slices, stored as 8 copies shifted by r = 0..7 elements so that
// every 16-byte chunk of a Toeplitz tile row is one aligned load.
// Block 2 tc_nch: W2 = sum phi_l w_l^2 (strided partial sums, then a fixed
// tree).  256 threads.
__device__ __forceinline__ void tc_filter_body(const Geom& g, const FastView& f, int b) {
    __shared__ float sl[kSl][256];
    __shared__ double red[256];
    const int i = threadIdx.x;
    if (b == 2 * f.tc_nch) {
        double s = 0.0;
        for (int64_t l = threadIdx.x; l < g.n_w; l += blockDim.x) {
            const double w = (double)(l - g.hw) * g.delta;
            s += f.phi[l] * (w * w);
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) *f.W2_dev = red[0];
        return;
    }
    const int c = b % f.tc_nch, flt = b / f.tc_nch;
    const int64_t l = (int64_t)kTcK * c - 127 + i;
    double h = 0.0;
    if (l >= 0 && l < g.n_w) {
        h = f.phi[l];
        if (flt == 0) h = h * ((double)(l - g.hw) * g.delta);
    }
    red[i] = fabs(h);
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (i < s) red[i] = fmax(red[i], red[i + s]);
        __syncthreads();
    }
    int e = 0;
    if (red[0] > 0.0) frexp(red[0], &e);   // 2^e > max |h|
    double v = ldexp(h, -e);
#pragma unroll
    for (int t = 0; t < kSl; ++t) {
        const double s = rint(v * 256.0);
        v = v * 256.0 - s;   // exact
        sl[t][i] = (float)s;
    }
    __syncthreads();
    uint16_t* out = f.tc_h + (size_t)(flt * f.tc_nch + c) * kSl * 8 * 256;
    for (int t = 0; t < kSl; ++t)
        for (int r = 0; r < 8; ++r)
            out[((size_t)t * 8 + r) * 256 + i] = bf16_bits(i + r < 256 ? sl[t][i + r] : 0.f);
    if (i == 0) f.tc_he[flt * f.tc_nch + c] = e;
}

__global__ void __launch_bounds__(256) k_tc_filter(Geom g, FastView f) {
    tc_filter_body(g, f, blockIdx.x);
}

__global__ void __launch_bounds__(256) kb_tc_filter(const SetupDev* descs,
                                                   const BlockRef* map) {
    const BlockRef r = map[blockIdx.x];
    const SetupDev& d = descs[r.inst];
    tc_filter_body(d.g, d.f, r.local);
}

// ---- E and the signal slices (every sweep) ------------------------------

// Block bx: E-indices m = 128 bx + j.  E_m = U^(y_{jlo+m}) - y (U constant
// beyond the table) in double-float for the second screening tier; the three
// signals E, E^2 = E_m E_m and E E_+ = E_m E_{m+1} (FP64 products) as
// double-float, scaled by the block's power of two and cut into slices.  Ud
// for the serial costs rides along on the same blocks.
__device__ __forceinline__ void build_E_tc_body(const Geom& g, const FastView& f,
                                                const double* __restrict__ U,
                                                double* __restrict__ Ud, int64_t bx) {
    __shared__ float wmax[3][4];
    const int j = threadIdx.x;
    const int64_t m = bx * 128 + j;
    if (m < g.n_y) Ud[m] = m + 1 < g.n_y ? __dsub_rn(U[m + 1], U[m]) : 0.0;
    dfloat x[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (m < f.n_e) {
        const int64_t jj = f.jlo + m;
        const int64_t a = jj < 0 ? 0 : (jj > g.n_y - 1 ? g.n_y - 1 : jj);
        const int64_t b = jj + 1 < 0 ? 0 : (jj + 1 > g.n_y - 1 ? g.n_y - 1 : jj + 1);
        const double e0 = U[a] - (double)(jj - g.hy) * g.delta;
        const double e1 = U[b] - (double)(jj + 1 - g.hy) * g.delta;
        x[0] = df_from_double(e0);
        x[1] = df_from_double(e0 * e0);
        x[2] = df_from_double(e0 * e1);
        f.E[m] = x[0];
    }
    if (bx >= f.tc_nblk) return;   // uniform over the block
    float mx[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        mx[s] = fabsf(x[s].hi);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            mx[s] = fmaxf(mx[s], __shfl_xor_sync(0xffffffffu, mx[s], off));
        if ((j & 31) == 0) wmax[s][j >> 5] = mx[s];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const float M = fmaxf(fmaxf(wmax[s][0], wmax[s][1]), fmaxf(wmax[s][2], wmax[s][3]));
        int e = 0;
        if (M > 0.f) frexpf(M, &e);   // 2^e > max |hi|, hence > |hi + lo|
        float rh = ldexpf(x[s].hi, -e), rl = ldexpf(x[s].lo, -e);
        uint16_t* out = f.tc_x + ((size_t)s * kSl * f.tc_nblk + bx) * 128 + j;
#pragma unroll
        for (int t = 0; t < kSl; ++t) {
            const float y = rh * 256.f, z = rl * 256.f;   // exact
            const float st = rintf(y);
            const float d = __fsub_rn(y, st);              // exact
            two_sum(d, z, rh, rl);                         // exact
            out[(size_t)t * f.tc_nblk * 128] = bf16_bits(st);
        }
        if (j == 0) f.tc_xe[s * f.tc_nblk + bx] = e;
    }
}

__global__ void __launch_bounds__(128) k_build_E_tc(Geom g, FastView f,
                                                     const double* __restrict__ U,
                                                     double* __restrict__ Ud) {
    build_E_tc_body(g, f, U, Ud, blockIdx.x);
}

// ---- the slice products on the tensor cores ------------------------------

struct TcShared {
    uint64_t full[kTcABuf];    // filter tile of slice group s built: full[s % kTcABuf]
    uint64_t empty[kTcABuf];   // MMAs of slice group s done: empty[s % kTcABuf]
    uint64_t bar_x[kTcSlices];   // signal tile of slice t landed (TMA)
    uint64_t bar_h;    // filter slices landed (bulk copy)
    uint64_t drain;    // every MMA issued so far done (error path)
    uint32_t tmem;
};

// Warp 0 issues the MMAs (one elected thread); warps 1 .. kTcT / 32 - 1 build
// the filter tiles into the ring.
constexpr int kTcBuilders = kTcT - 32;

// Test hook 2 (kept out of the pipeline's code): the builders fill only the
// first filter buffer; the MMA thread issues slice group 0, its wait for the
// second tile runs out after the short bound, and it waits for the issued
// MMAs (drain barrier) before returning.  Leaves nothing in flight.
__device__ __noinline__ void tc_hook_one_group(char* tA, const char* tB, const char* tH,
                                               uint32_t tmem, TcShared& ts) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp > 0) {
        for (int k = tid - 32; k < 128 * 16; k += kTcBuilders) {
            const int b = k >> 4, jc = k & 15;
            const int r = 7 - (b & 7);
            const int q = jc + 15 - (b >> 3);
            *(uint4*)(tA + sw128_offset(128, b, jc)) = *(const uint4*)(tH + (r * 256 + 8 * q) * 2);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ts.full[0]);
        return;
    }
    if (lane != 0) return;
    if (!mbar_wait(&ts.full[0], 0, kTcPolls)) return;
    tc_fence_after();
    constexpr uint32_t idesc = umma_idesc_bf16(128, 64);
    const uint32_t a0 = smem_u32(tA);
    bool issued = false;
    for (int t = 0; t < kSl; ++t) {
        if (!mbar_wait(&ts.bar_x[t], 0, kTcPolls)) break;
        const uint32_t b0 = smem_u32(tB + t * kTcBTile);
        for (int kk = 0; kk < 8; ++kk) {
            const uint32_t off = (uint32_t)((kk & 3) * 32);
            umma_bf16(tmem + (uint32_t)(t * 64),
                      umma_desc_sw128(a0 + (kk >> 2) * (128 * 128) + off),
                      umma_desc_sw128(b0 + (kk >> 2) * (64 * 128) + off), idesc,
                      kk > 0 ? 1u : 0u);
        }
        issued = true;
    }
    mbar_wait(&ts.full[1], 0, kTcHookPolls);   // never filled: runs out
    if (issued) {
        umma_commit(&ts.drain);
        mbar_wait(&ts.drain, 0, kTcPolls);
    }
}

// Table tau (0: P from E and a; 1: Q from E^2 and phi; 2: R from E E_+ and
// phi), column group grp (columns a = 64 grp .. + 63), tap chunk c: the
// double-float partial D_c[b][a] of positions 128 a + b into tc_part.
// `tmap` is the signal's TMA map (kernel parameter or global memory).
//
// Pipeline: slice group s (filter slice s against signal slices t < kSl - s,
// accumulator s + t) reads filter buffer s % kTcABuf.  The builder warps fill
// a buffer once the group that last read it is done (empty, committed by the
// MMA thread) and arrive on its full barrier; the MMA thread waits on full,
// issues the group and commits it to empty.  No block-wide barrier between
// groups: the tensor core runs while the next tiles are built.  The j-th use
// of a buffer is its barriers' phase j (parity j & 1); a builder never runs
// more than one phase ahead of the MMA thread, so parities cannot alias.
__device__ __forceinline__ void tc_tables_body(const FastView& f, const CUtensorMap* tmap,
                                               int tau, int grp, int c, char* smem_raw,
                                               TcShared& ts) {
    char* base = (char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    char* tB = base;                     // kSl signal tiles (all slices)
    char* tA = base + kSl * kTcBTile;    // kTcABuf filter tiles (ring)
    char* tH = tA + kTcABuf * kTcATile;  // the chunk's filter slices, 8 shifts each
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int flt = tau == 0 ? 0 : 1;
    const int hook_kind = f.tc_err[1];    // test hook (see kTcHookPolls)
    const bool hook = hook_kind == 1;     // the filter copy is not issued
    if (tid == 0) {
        for (int k = 0; k < kTcABuf; ++k) {
            mbar_init(&ts.full[k], kTcBuilders / 32);
            mbar_init(&ts.empty[k], 1);
        }
        for (int t = 0; t < kSl; ++t) mbar_init(&ts.bar_x[t], 1);
        mbar_init(&ts.bar_h, 1);
        mbar_init(&ts.drain, 1);
        fence_mbar_init();
        // filter slices of the chunk (contiguous), then the signal tiles: row
        // r of slice t is block 64 grp + r + c, two 64-wide boxes per slice
        if (!hook) {
            mbar_expect_tx(&ts.bar_h, kTcHBytes);
            bulk_load(tH, f.tc_h + (size_t)(flt * f.tc_nch + c) * kSl * 8 * 256, kTcHBytes,
                      &ts.bar_h);
        }
        const int row0 = 64 * grp + c;
        for (int t = 0; t < kSl; ++t) {
            const int y = (int)(t * f.tc_nblk) + row0;
            mbar_expect_tx(&ts.bar_x[t], kTcBTile);
            tma_load_2d(tB + t * kTcBTile, tmap, 0, y, &ts.bar_x[t]);
            tma_load_2d(tB + t * kTcBTile + 64 * 128, tmap, 64, y, &ts.bar_x[t]);
        }
    }
    if (warp == 0) tmem_alloc(&ts.tmem, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // filter tile of slice s: row b holds G[m - b + 127], m < 128 (builder
    // thread bt of kTcBuilders)
    auto build_A = [&](int s, char* dst, int bt) {
        const char* hs = tH + (size_t)s * 8 * 256 * 2;
        for (int k = bt; k < 128 * 16; k += kTcBuilders) {
            const int b = k >> 4, jc = k & 15;
            const int r = 7 - (b & 7);
            const int q = jc + 15 - (b >> 3);
            *(uint4*)(dst + sw128_offset(128, b, jc)) =
                *(const uint4*)(hs + (r * 256 + 8 * q) * 2);
        }
    };
    bool ok = mbar_wait(&ts.bar_h, 0, hook ? kTcHookPolls : kTcPolls);
    ok = __syncthreads_and(ok);
    const uint32_t tmem = ts.tmem;
    constexpr uint32_t idesc = umma_idesc_bf16(128, 64);
    if (ok && hook_kind == 2) {
        tc_hook_one_group(tA, tB, tH, tmem, ts);
        ok = false;
    } else if (ok && warp == 0) {
        if (lane == 0) {
            bool issued = false;
            for (int s = 0; s < kSl && ok; ++s) {
                ok = mbar_wait(&ts.full[s % kTcABuf], (s / kTcABuf) & 1, kTcPolls);
                if (!ok) break;
                tc_fence_after();
                const uint32_t a0 = smem_u32(tA + (s % kTcABuf) * kTcATile);
                for (int t = 0; s + t < kSl; ++t) {
                    // the first slice group starts as the signal tiles land
                    if (s == 0) ok = mbar_wait(&ts.bar_x[t], 0, kTcPolls);
                    if (!ok) break;
                    const uint32_t b0 = smem_u32(tB + t * kTcBTile);
                    const uint32_t d = tmem + (uint32_t)((s + t) * 64);
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint32_t off = (uint32_t)((kk & 3) * 32);
                        umma_bf16(d, umma_desc_sw128(a0 + (kk >> 2) * (128 * 128) + off),
                                  umma_desc_sw128(b0 + (kk >> 2) * (64 * 128) + off), idesc,
                                  (s > 0 || kk > 0) ? 1u : 0u);
                    }
                    issued = true;
                }
                if (!ok) break;
                umma_commit(&ts.empty[s % kTcABuf]);
            }
            if (!ok && issued) {
                // drain what was issued before tensor memory is freed
                umma_commit(&ts.drain);
                mbar_wait(&ts.drain, 0, kTcPolls);
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
    } else if (ok) {
        const int bt = tid - 32;
        for (int s = 0; s < kSl && ok; ++s) {
            char* dst = tA + (s % kTcABuf) * kTcATile;
            if (s >= kTcABuf) {
                // the group that read this buffer last is done
                ok = mbar_wait(&ts.empty[s % kTcABuf], ((s - kTcABuf) / kTcABuf) & 1,
                               kTcPolls);
                ok = __all_sync(0xffffffffu, ok);   // the warp stays together
                if (!ok) break;
                fence_proxy_async_smem();   // the tensor core's reads before our writes
            }
            build_A(s, dst, bt);
            fence_proxy_async_smem();       // our writes before the tensor core's reads
            __syncwarp();
            if (lane == 0) mbar_arrive(&ts.full[s % kTcABuf]);
        }
    }
    // the last commit covers every MMA
    if (ok)
        ok = mbar_wait(&ts.empty[(kSl - 1) % kTcABuf], ((kSl - 1) / kTcABuf) & 1, kTcPolls);
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (ok) {
        const int qd = warp & 3, col0 = 16 * (warp >> 2);
        const int b = 32 * qd + lane;
        const uint32_t lbase = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)col0;
        const int he = f.tc_he[flt * f.tc_nch + c];
        const int32_t* xe = f.tc_xe + (size_t)tau * f.tc_nblk;
        float2* part = f.tc_part + (size_t)(tau * f.tc_nch + c) * f.tc_ng * 64 * 128;
        float v[16], w[16];
        dfloat acc[16];
        // D_5 2^-40 + D_4 2^-32 in FP32 (one rounding of a sum below
        // 2^-23.7 sigma_h sigma_x 2^16), then D_3 .. D_0 in double-float,
        // smallest first
        tmem_ld16(lbase + 5 * 64, v);
        tmem_ld16(lbase + 4 * 64, w);
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = {__fmaf_rn(w[e], 0x1p-32f, v[e] * 0x1p-40f), 0.f};
#pragma unroll 1
        for (int k = 3; k >= 0; --k) {
            tmem_ld16(lbase + (uint32_t)(k * 64), v);
            const float sc = __int_as_float((127 - 8 * k) << 23);
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[e] = df_add_f(acc[e], v[e] * sc);
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int64_t a = (int64_t)64 * grp + col0 + e;
            const int ex = he + xe[a + c] - 16;
            float2 o;
            if (ex >= -126 && ex <= 127) {
                const float sc = __int_as_float((ex + 127) << 23);
                o = make_float2(acc[e].hi * sc, acc[e].lo * sc);
            } else {
                o = make_float2(ldexpf(acc[e].hi, ex), ldexpf(acc[e].lo, ex));
            }
            part[a * 128 + b] = o;
        }
    } else {
        // A wait gave up: the signal copies this CTA issued land before it
        // exits (bounded waits; completed phases return at once), and zero
        // partials keep the kernels after it on finite values.
        if (tid == 0) {
            atomicExch(f.tc_err, 1);
            for (int t = 0; t < kSl; ++t) mbar_wait(&ts.bar_x[t], 0, kTcPolls);
        }
        const int col0 = 16 * (warp >> 2), b = 32 * (warp & 3) + lane;
        float2* part = f.tc_part + (size_t)(tau * f.tc_nch + c) * f.tc_ng * 64 * 128;
        for (int e = 0; e < 16; ++e)
            part[((int64_t)64 * grp + col0 + e) * 128 + b] = make_float2(0.f, 0.f);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

__global__ void __launch_bounds__(kTcT, 1) k_tc_tables(const __grid_constant__ FastView f) {
    extern __shared__ char tc_smem[];
    __shared__ TcShared ts;
    const int per = f.tc_ng * f.tc_nch;
    const int tau = blockIdx.x / per, rest = blockIdx.x % per;
    tc_tables_body(f, &f.tc_map[tau], tau, rest / f.tc_nch, rest % f.tc_nch, tc_smem, ts);
}

// ---- chunk sums and the error bound ---------------------------------------

constexpr int kCombT = 384;   // three tables x 128 positions
constexpr int kCombBatch = 24; // chunk partials loaded at once per thread

// Column a (128 positions); thread (tau, b): table tau at p = 128 a + b as the
// chunk partials added in a fixed order (four interleaved chains, then
// pairwise) by accurate double-float additions (df_add_acc: |error| <=
// 3 u^2 |result|, u = 2^-24), and tc_bt[a], a bound
// on the error of the table identity's S at any cell whose two positions lie
// in column a: 2 max_p beta_P(p) + max_p max(beta_Q(p), beta_R(p)) with, per
// table,
//   beta(p) = 1.25 [1.25 2^-39 sum_c 2^(he(c) + xe(a + c)) slices, products, fold
//                   + 3.01 u^2 sum over additions |result|  chunk additions
//                   + 2^-130]                              underflow of scaled lows
// The first term: per product term 3.32 2^-48 sigma_h sigma_x (double-float
// and FP64 rounding of the signal 2^-48 + 2^-53, slice truncations 2 x 2^-49,
// FP64 a_l 2^-53, dropped products s + t >= 6 1.26 2^-48), 128 terms per chunk,
// plus 142 2^-48 sigma_h sigma_x for folding the six accumulators (the two
// smallest in FP32: <= 1.2 2^-48; then smallest first in double-float,
// df_add_f error <= u^2 (2 |a| + |b|): <= 141 2^-48): 567 2^-48 <= 1.25 2^-39
// per chunk.
__device__ __forceinline__ void tc_combine_body(const FastView& f, int64_t a) {
    __shared__ float colterm[3];
    __shared__ float wmax[kCombT / 32];
    const int tid = threadIdx.x, tau = tid >> 7, b = tid & 127;
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t p = a * 128 + b;
    if (b < 32) {   // the slice term of this table and column
        const int flt = tau == 0 ? 0 : 1;
        float sum = 0.f;
        for (int c = lane; c < f.tc_nch; c += 32)
            sum += ldexpf(1.f, f.tc_he[flt * f.tc_nch + c] +
                                   f.tc_xe[(size_t)tau * f.tc_nblk + a + c] - 39);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        if (lane == 0) colterm[tau] = 1.25f * sum * 1.0001f;
    }
    const size_t stride = (size_t)f.tc_ng * 64 * 128;
    const float2* part = f.tc_part + (size_t)tau * f.tc_nch * stride + p;
    // four interleaved chains (chunk c into chain c % 4), then
    // (chain 0 + chain 1) + (chain 2 + chain 3)
    dfloat ch[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    float mag = 0.f;
    for (int c0 = 0; c0 < f.tc_nch; c0 += kCombBatch) {
        float2 v[kCombBatch];
#pragma unroll
        for (int k = 0; k < kCombBatch; ++k)   // issue the loads, then add in order
            v[k] = c0 + k < f.tc_nch ? __ldcg(part + (size_t)(c0 + k) * stride)
                                     : make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < kCombBatch; ++k)
            if (c0 + k < f.tc_nch) {
                dfloat& a = ch[k & 3];   // kCombBatch is a multiple of 4
                a = df_add_acc(a, dfloat{v[k].x, v[k].y});
                mag += fabsf(a.hi);
            }
    }
    const dfloat s01 = df_add_acc(ch[0], ch[1]), s23 = df_add_acc(ch[2], ch[3]);
    const dfloat r = df_add_acc(s01, s23);
    mag += fabsf(s01.hi) + fabsf(s23.hi) + fabsf(r.hi);
    dfloat* out = tau == 0 ? f.P : (tau == 1 ? f.Q : f.R);
    if (p < f.n_pos) out[p] = r;
    __syncthreads();
    float beta = p < f.n_pos ? 1.25f * (colterm[tau] + 3.01f * 0x1p-48f * mag * 1.0001f +
                                        0x1p-130f)
                             : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) beta = fmaxf(beta, __shfl_xor_sync(0xffffffffu, beta, off));
    if (lane == 0) wmax[warp] = beta;
    __syncthreads();
    if (tid == 0) {
        float mp = 0.f, mq = 0.f;
        for (int w = 0; w < 4; ++w) mp = fmaxf(mp, wmax[w]);
        for (int w = 4; w < kCombT / 32; ++w) mq = fmaxf(mq, wmax[w]);
        f.tc_bt[a] = (2.f * mp + mq) * 1.0001f;
    }
}

__global__ void __launch_bounds__(kCombT) k_tc_combine(FastView f) {
    tc_combine_body(f, blockIdx.x);
}

// ---- batched wrappers -------------------------------------------------------

__device__ __forceinline__ BlockRef stage_tc(const InstDev* insts, const BlockRef* map,
                                             InstDev& sd) {
    const BlockRef r = map[blockIdx.x];
    const int* src = (const int*)(insts + r.inst);
    int* dst = (int*)&sd;
    for (int k = threadIdx.x; k < (int)(sizeof(InstDev) / 4); k += blockDim.x)
        dst[k] = src[k];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(128) kb_build_E_tc(const InstDev* insts,
                                                     const BlockRef* map) {
    __shared__ InstDev sd;
    const BlockRef r = stage_tc(insts, map, sd);
    build_E_tc_body(sd.g, sd.f, sd.U, sd.Ud, r.local);
}

__global__ void __launch_bounds__(kTcT, 1) kb_tc_tables(const InstDev* insts,
                                                        const BlockRef* map) {
    extern __shared__ char tc_smem[];
    __shared__ InstDev sd;
    __shared__ TcShared ts;
    const BlockRef r = stage_tc(insts, map, sd);
    const int per = sd.f.tc_ng * sd.f.tc_nch;
    const int tau = r.local / per, rest = r.local % per;
    const CUtensorMap* tmap = &insts[r.inst].f.tc_map[tau];   // global memory
    if (threadIdx.x == 0) tmap_acquire(tmap);
    tc_tables_body(sd.f, tmap, tau, rest / sd.f.tc_nch, rest % sd.f.tc_nch, tc_smem, ts);
}

__global__ void __launch_bounds__(kCombT) kb_tc_combine(const InstDev* insts,
                                                     const BlockRef* map) {
    __shared__ InstDev sd;
    const BlockRef r = stage_tc(insts, map, sd);
    tc_combine_body(sd.f, r.local);
}

}  // namespace

// ---- host side --------------------------------------------------------------

void tc_plan(const Geom& g, FastPlan* fp) {
    fp->tc_na = (fp->n_pos + 127) / 128;
    fp->tc_ng = (int)((fp->tc_na + 63) / 64);
    fp->tc_nch = (int)((g.n_w + 127 + kTcK - 1) / kTcK);
    fp->tc_nblk = (int64_t)64 * fp->tc_ng + fp->tc_nch - 1;
}

size_t tc_bytes(const FastPlan& fp, size_t align, size_t* sizes) {
    sizes[0] = (size_t)2 * fp.tc_nch * kSl * 8 * 256 * 2;       // tc_h
    sizes[1] = (size_t)2 * fp.tc_nch * 4;                       // tc_he
    sizes[2] = (size_t)3 * kSl * fp.tc_nblk * 128 * 2;          // tc_x
    sizes[3] = (size_t)3 * fp.tc_nblk * 4;                      // tc_xe
    sizes[4] = (size_t)3 * fp.tc_nch * fp.tc_ng * 64 * 128 * 8; // tc_part
    sizes[5] = (size_t)(fp.tc_na + 1) * 4;                      // tc_bt
    sizes[6] = 8;                                               // tc_err, test hook
    size_t total = 0;
    for (int k = 0; k < 7; ++k) total += (sizes[k] + align - 1) / align * align;
    return total;
}

bool tc_encode_maps(FastView* f) {
    static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> encode{nullptr};
    if (!encode.load()) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode.store((PFN_cuTensorMapEncodeTiled_v12000)fn);
    }
    for (int sig = 0; sig < 3; ++sig) {
        void* base = f->tc_x + (size_t)sig * kSl * f->tc_nblk * 128;
        const cuuint64_t dims[2] = {128, (cuuint64_t)kSl * (cuuint64_t)f->tc_nblk};
        const cuuint64_t strides[1] = {256};
        const cuuint32_t box[2] = {64, 64};
        const cuuint32_t estr[2] = {1, 1};
        if (encode.load()(&f->tc_map[sig], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

int64_t tc_build_E_blocks(const Geom& g, const FastPlan& fp) {
    int64_t n = fp.tc_nblk * 128;
    if (fp.n_e > n) n = fp.n_e;
    if (g.n_y > n) n = g.n_y;
    return (n + 127) / 128;
}

int64_t tc_table_blocks(const FastPlan& fp) { return (int64_t)3 * fp.tc_ng * fp.tc_nch; }

int64_t tc_combine_blocks(const FastPlan& fp) { return fp.tc_na; }

cudaError_t tc_init_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_tc_tables, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kb_tc_tables, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kTcSmem);
}

void launch_tc_setup(const Geom& g, const FastView& f, cudaStream_t s) {
    k_tc_filter<<<(unsigned)(2 * f.tc_nch + 1), 256, 0, s>>>(g, f);
}

void launch_batch_setup_tc(const SetupLaunch& sl, cudaStream_t s) {
    if (sl.filter_blocks)
        kb_tc_filter<<<(unsigned)sl.filter_blocks, 256, 0, s>>>(sl.descs, sl.filter_map);
}

void launch_tables(const Geom& g, const FastView& f, const double* U, double* Ud,
                   cudaStream_t s, Prof* prof) {
    cudaEvent_t ev;
    int k = prof ? prof->begin("build_E", &ev) : -1;
    k_build_E_tc<<<(unsigned)tc_build_E_blocks(g, f), 128, 0, s>>>(g, f, U, Ud);
    if (prof) prof->end(k, ev);
    k = prof ? prof->begin("tables", &ev) : -1;
    k_tc_tables<<<(unsigned)tc_table_blocks(f), kTcT, kTcSmem, s>>>(f);
    if (prof) prof->end(k, ev);
    k = prof ? prof->begin("tab_combine", &ev) : -1;
    k_tc_combine<<<(unsigned)tc_combine_blocks(f), kCombT, 0, s>>>(f);
    if (prof) prof->end(k, ev);
}

void launch_batch_tables(const BatchLaunch& bl, cudaStream_t s, Prof* prof) {
    const InstDev* d = bl.insts;
    {
        ProfScope ps(prof, "build_E");
        kb_build_E_tc<<<(unsigned)bl.n_blocks[kBBuildE], 128, 0, s>>>(d, bl.map[kBBuildE]);
    }
    {
        ProfScope ps(prof, "tables");
        kb_tc_tables<<<(unsigned)bl.n_blocks[kBTabPart], kTcT, kTcSmem, s>>>(d, bl.map[kBTabPart]);
    }
    ProfScope ps(prof, "tab_combine");
    kb_tc_combine<<<(unsigned)bl.n_blocks[kBTabComb], kCombT, 0, s>>>(d, bl.map[kBTabComb]);
}

}  // namespace ucp
