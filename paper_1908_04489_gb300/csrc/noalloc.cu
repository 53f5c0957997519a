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
constexpr int kMaxTiles = 8;           // source tiles of the u1 step

constexpr size_t rnd256(size_t n) { return (n + 255) / 256 * 256; }
// nu and prior (x-sized), the constant table, then the u1 buffers at the
// largest sizes: src_nu, src_f, src_F; per tile the box count, per box slot
// its first source, size, geometry, range, exp(delta c) and 2 kBoxTerms
// coefficients; per tile the partial moments of its 32-source chunks (at
// most tile / 32 + kBoxMax, tiles of at most kMaxX / kMaxTiles sources);
// per run (at most n_y runs) two bounds; per tile and target the numerator
// and denominator partials.
constexpr size_t kSlots = (size_t)kMaxTiles * kBoxMax;
constexpr size_t kChunks = (size_t)kMaxTiles * (kMaxX / kMaxTiles / 32 + kBoxMax);
constexpr size_t kScratchBytes =
    5 * rnd256(8 * kMaxX) + rnd256(8 * kConstTab) + rnd256(4 * kMaxTiles) +
    2 * rnd256(4 * kSlots) + 2 * rnd256(16 * kSlots) + rnd256(8 * kSlots) +
    rnd256(8 * kSlots * 2 * kBoxTerms) + rnd256(8 * kChunks * (kBoxTerms + 1)) +
    2 * rnd256(4 * kMaxY) + 2 * rnd256(8 * (size_t)kMaxTiles * kMaxY);

static __device__ __align__(256) double g_scratch[kScratchBytes / 8];

// Bump allocation from the static array (256-byte steps).
struct Bump {
    char* p;
    char* end;
};
static void* bump_get(void* ctx, size_t n) {
    Bump* b = (Bump*)ctx;
    n = rnd256(n);
    if ((size_t)(b->end - b->p) < n) return nullptr;
    void* r = b->p;
    b->p += n;
    return r;
}

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
    if (k < kConstTab) t64[k] = const_table_entry((int)k);
}

// Device address of g_scratch on the current device.  Outside stream
// capture it is looked up on every call (a context torn down by
// cudaDeviceReset reloads the module at another address); while `stream` is
// capturing, the address of the last uncaptured call on this device is used
// (a symbol lookup may load the module, which capture forbids).
static ucp_status scratch_address(cudaStream_t stream, double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        set_error("ucp_u1_update_noalloc: %s%s", "no current CUDA device", "");
        return UCP_E_CUDA;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusNone;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap != cudaStreamCaptureStatusNone && !g_addr[dev]) {
        set_error("ucp_u1_update_noalloc: %s%s",
                  "first call on this device made during stream capture", "");
        return UCP_E_STATE;
    }
    if (cap == cudaStreamCaptureStatusNone) {
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
    if (g.problem != 0) {
        set_error("ucp_u1_update_noalloc: %s%s", "Witsenhausen's problem (problem 0) only", "");
        return UCP_E_ARG;
    }
    if (g.n_x > kMaxX || g.n_y > kMaxY) {
        set_error("ucp_u1_update_noalloc: %s%s",
                  "grid too large for the static scratch (needs n_x <= 32768 "
                  "and n_y <= 32768)", "");
        return UCP_E_ARG;
    }
    double* base = nullptr;
    ucp_status st = scratch_address((cudaStream_t)stream, &base);
    if (st != UCP_OK) return st;

    // plan of the u1 kernels over at most kMaxTiles source tiles
    FastView f{};
    u1_plan(g, kMaxTiles, &f);
    const dfloat sd = df_from_double(ldexp(g.delta, -g.shift));
    f.step_hi = sd.hi;
    f.step_lo = sd.lo;
    const dfloat dd = df_from_double(g.delta);
    f.delta_hi = dd.hi;
    f.delta_lo = dd.lo;

    Bump bump{(char*)base, (char*)base + kScratchBytes};
    int64_t* nu = (int64_t*)bump_get(&bump, 8 * (size_t)g.n_x);
    f.prior = (dfloat*)bump_get(&bump, 8 * (size_t)g.n_x);
    f.t64 = (dfloat*)bump_get(&bump, 8 * kConstTab);
    if (!nu || !f.prior || !f.t64 || !u1_carve(g, &f, bump_get, &bump)) {
        set_error("ucp_u1_update_noalloc: %s%s", "static scratch too small", "");
        return UCP_E_ARG;
    }

    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g.n_x > kConstTab ? g.n_x : kConstTab;
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
