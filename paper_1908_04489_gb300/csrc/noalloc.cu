// noalloc.cu -- ucp_u1_update_noalloc: the u1 step (U_j = E[x1 | y1 = y_j])
// for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- a host
// process whose device memory is owned and budgeted by another framework, a
// real-time control loop that must not enter the allocator (its latency and
// failure modes are not bounded), or a plug-in that is handed only the
// buffers it reads and writes.  Such callers pass the input controller and
// the output table; every intermediate buffer of the u1 kernels lives in one
// file-scope device array of fixed size, set aside in every GPU that loads
// the library until the process exits.
//
// Limits: n_x <= kMaxX and n_y <= kMaxY (grid sizes of ucp_params); larger
// problems are rejected with UCP_E_ARG.  The first call on a device looks up
// the array's device address (cudaGetSymbolAddress) with that device
// current; make that first call before any stream capture.  All calls share
// the one array, so calls whose work overlaps on the GPU (other streams,
// other host threads) race; serialise them.  Every scratch entry a call
// reads is written earlier in the same call, so nothing needs clearing.
#include <math.h>

#include <mutex>

#include "ucp_fast.cuh"

namespace ucp {
void set_error(const char* fmt, const char* a, const char* b);
}

namespace {

using namespace ucp;

constexpr int64_t kMaxX = 32768;       // largest x0 grid
constexpr int64_t kMaxY = 32768;       // largest y grid
constexpr int kMaxChunks = 8;          // source columns of the u1 kernel
constexpr int kThreadsPerRow = 64;     // threads per block row (k_mmse_main)

// 8-byte slots: nu, prior, src_nu, src_f, src_F (x-sized); mshift, psi
// (y-sized); the exp(k/64) table; numerator and denominator partials; the
// per-chunk exponent minima (floats, two per slot).
constexpr size_t kScratchDoubles = 5 * (size_t)kMaxX + 2 * (size_t)kMaxY + 64 +
                                   2 * (size_t)kMaxChunks * kMaxY +
                                   (size_t)kMaxChunks * kMaxY / 2;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
static std::mutex g_mu;
static double* g_addr[kMaxDevices] = {};

__global__ void k_na_prepare(Geom g, const double* __restrict__ f,
                             int64_t* __restrict__ nu, dfloat* __restrict__ prior,
                             dfloat* __restrict__ t64) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < g.n_x) {
        const double v = __dmul_rn(__ddiv_rn(f[k], g.delta), (double)g.one);
        nu[k] = llround(v);
        const double x = __dmul_rn((double)(k - g.hx), g.delta);
        prior[k] = df_from_double(__ddiv_rn(__dmul_rn(x, x), g.two_s2));
    }
    if (k < 47) t64[k] = df_from_double(exp((double)(k - 23) / 64.0));
}

// Device address of g_scratch on the current device (looked up once).
static ucp_status scratch_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        set_error("ucp_u1_update_noalloc: %s%s", "no current CUDA device", "");
        return UCP_E_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error("ucp_u1_update_noalloc: cudaGetSymbolAddress failed: %s%s",
                      cudaGetErrorString(e), "");
            return UCP_E_CUDA;
        }
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return UCP_OK;
}

}  // namespace

extern "C" UCP_API ucp_status ucp_u1_update_noalloc(const ucp_params* params,
                                                    const double* f_dev,
                                                    double* u1_dev,
                                                    void* stream) {
    if (!params || !f_dev || !u1_dev) {
        set_error("ucp_u1_update_noalloc: %s%s", "NULL argument", "");
        return UCP_E_ARG;
    }
    Geom g;
    if (const char* why = make_geom(*params, &g)) {
        set_error("ucp_u1_update_noalloc: %s%s", why, "");
        return UCP_E_ARG;
    }
    if (g.n_x > kMaxX || g.n_y > kMaxY) {
        set_error("ucp_u1_update_noalloc: %s%s",
                  "grid too large for the static scratch (needs n_x <= 32768 "
                  "and n_y <= 32768)", "");
        return UCP_E_ARG;
    }
    double* base = nullptr;
    ucp_status st = scratch_address(&base);
    if (st != UCP_OK) return st;

    // plan of the u1 kernels over at most kMaxChunks source columns
    FastView f{};
    f.run = mmse_run_length(g);
    const int64_t per_row = (int64_t)kThreadsPerRow * f.run;
    f.j_blocks = (g.n_y + per_row - 1) / per_row;
    int64_t chunks = (4 * 152 + f.j_blocks - 1) / f.j_blocks;
    if (chunks > kMaxChunks) chunks = kMaxChunks;
    const int64_t max_chunks = (g.n_x + 127) / 128;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    f.chunk = ((g.n_x + chunks - 1) / chunks + 63) / 64 * 64;
    f.n_chunks = (int)((g.n_x + f.chunk - 1) / f.chunk);
    const dfloat sd = df_from_double(ldexp(g.delta, -g.shift));
    f.step_hi = sd.hi;
    f.step_lo = sd.lo;

    double* q = base;
    int64_t* nu = (int64_t*)q;  q += kMaxX;
    f.prior = (dfloat*)q;       q += kMaxX;
    f.src_nu = (int64_t*)q;     q += kMaxX;
    f.src_f = (dfloat*)q;       q += kMaxX;
    f.src_F = (dfloat*)q;       q += kMaxX;
    f.mshift = (float*)q;       q += kMaxY;
    f.psi = (dfloat*)q;         q += kMaxY;
    f.t64 = (dfloat*)q;         q += 64;
    f.partN = q;                q += (size_t)kMaxChunks * kMaxY;
    f.partD = q;                q += (size_t)kMaxChunks * kMaxY;
    f.mshift_part = (float*)q;

    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g.n_x > 47 ? g.n_x : 47;
    k_na_prepare<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, f_dev, nu, f.prior,
                                                          f.t64);
    launch_mmse_fast(g, f, nu, u1_dev, s, nullptr);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("ucp_u1_update_noalloc: %s%s", cudaGetErrorString(e), "");
        return UCP_E_CUDA;
    }
    return UCP_OK;
}
