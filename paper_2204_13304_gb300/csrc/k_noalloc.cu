// m2s_symgs_noalloc: symmetric Gauss-Seidel on the 27-point operator for
// callers that must not allocate device memory.
//
// Who needs it: host applications that reserve the whole device memory for
// their own pool up front (a cudaMalloc from this library would fail or
// fragment that pool), and latency-critical loops where the implicit
// device-wide synchronisation of cudaMalloc/cudaFree is not acceptable.
// They pass b and x, and this entry point allocates nothing: the scratch
// the sweeps need (the two old-neighbour-sum buffers, the unit tables, the
// progress counters and the status word) lives in one file-scope
// __device__ array of fixed size, created when the library is loaded and
// held by every GPU that loads it until the process exits.
//
// Limits: at most kMaxPoints = 2^18 grid points (64^3) and at most
// kMaxUnits wavefront units; larger requests are rejected with
// M2S_ERR_INVALID_ARG before anything is launched.
// Sharing: every call (on every stream) uses the same array, which keeps
// the last call's contents; the counters that must start at zero are
// cleared at the start of each call.  Calls that overlap on the GPU race on
// the array: serialise them (one stream, or synchronise between calls).
// Set-up: the first call on a device looks up the array's device address
// with cudaGetSymbolAddress (with that device current) and caches it; make
// that first call before any stream capture.
// Every call copies its unit tables from host memory, launches the sweeps on
// `stream`, synchronises `stream` and reads the status word back.  Its
// spin-waits are bounded by a fixed 4 s (m2s_set_spin_limit sets the bound
// of a grid and has no effect here).
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <new>
#include <vector>

#include "m2s_internal.cuh"

namespace m2s {
namespace {

constexpr i64 kMaxPoints = 1LL << 18;
constexpr int kMaxUnits = 8192;
constexpr long long kSpinNs = 4000000000LL;  // bound of every spin-wait
constexpr size_t kQBytes = (size_t)kMaxPoints * sizeof(double);  // one buffer
constexpr size_t kOriginOff = 2 * kQBytes;
constexpr size_t kProdOff = kOriginOff + (size_t)kMaxUnits * sizeof(int2);
constexpr size_t kFlagsOff = kProdOff + (size_t)kMaxUnits * sizeof(int4);
constexpr size_t kCtrlOff = kFlagsOff + (size_t)kMaxUnits * sizeof(int);
constexpr size_t kStatusOff = kCtrlOff + 256;
constexpr size_t kScratchBytes = kStatusOff + sizeof(DevStatus);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once).
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (unsigned char*)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

template <typename T>
cudaError_t run(Dims d, const T* b, T* x, int sweeps, unsigned char* base, const WaveUnits& u,
                DevStatus* status, cudaStream_t st) {
    T* Qa = (T*)base;
    T* Qb = (T*)(base + kQBytes);
    WaveCall c;
    c.publish_every = 4;
    c.spin_ns = kSpinNs;
    c.status = status;
    c.rz_partials = nullptr;
    c.stall_unit = -1;
    cudaError_t e = launch_st27<T>(ST27_QUP, d, d, x, nullptr, b, Qa, st);
    for (int s = 0; s < sweeps && e == cudaSuccess; ++s) {
        c.rev = 0;
        e = launch_gs27_wave<T>(u, c, d, Qa, Qb, b, x, st);
        if (e != cudaSuccess) break;
        c.rev = 1;
        e = launch_gs27_wave<T>(u, c, d, Qb, s + 1 < sweeps ? Qa : nullptr, b, x, st);
    }
    return e;
}

}  // namespace
}  // namespace m2s

using namespace m2s;

extern "C" m2s_status m2s_symgs_noalloc(int nx, int ny, int nz, m2s_dtype dtype, const void* b,
                                        void* x, int n_sym_sweeps, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !b || !x || b == x || n_sym_sweeps < 0)
        return M2S_ERR_INVALID_ARG;
    if (dtype != M2S_F64 && dtype != M2S_F32) return M2S_ERR_INVALID_ARG;
    const size_t align = dtype == M2S_F64 ? 8 : 4;
    if (((uintptr_t)b % align) != 0 || ((uintptr_t)x % align) != 0) return M2S_ERR_INVALID_ARG;
    const i64 n = (i64)nx * ny * nz;
    if (n > kMaxPoints) return M2S_ERR_INVALID_ARG;
    // b and x must not share a byte: the sweeps write x while reading b
    const uintptr_t bb = (uintptr_t)b, xb = (uintptr_t)x, bytes = (uintptr_t)n * align;
    if (bb < xb + bytes && xb < bb + bytes) return M2S_ERR_INVALID_ARG;
    if (n_sym_sweeps == 0) return M2S_OK;
    // Every row V of units (kWaveSlots - 1 planes of z) holds at least one
    // unit, so a grid with more such rows than kMaxUnits is rejected before
    // the host builds its unit table (whose index is (ny + nz) / 30 + 1 by
    // nz / 4 + 1 entries).
    const int slots = kWaveSlots - 1;
    if ((nz + slots - 1) / slots > kMaxUnits) return M2S_ERR_INVALID_ARG;
    Dims d{nx, ny, nz, n, 0};
    std::vector<int2> org;
    std::vector<int4> prod;
    try {
        build_units_host(30, 1, 1, kWaveSlots, d, org, prod);
    } catch (const std::bad_alloc&) {
        return M2S_ERR_OOM;
    }
    if ((int)org.size() > kMaxUnits) return M2S_ERR_INVALID_ARG;

    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return M2S_ERR_CUDA;
    WaveUnits u{};
    u.n_units = (int)org.size();
    u.K = kWaveSlots;
    u.stencil = 27;
    u.d_origin = (int2*)(base + kOriginOff);
    u.d_prod = (int4*)(base + kProdOff);
    u.d_flags = (int*)(base + kFlagsOff);
    u.d_ctrl = (int*)(base + kCtrlOff);
    u.grid = wave_grid(u.n_units, wave_blocks_per_sm(27));
    DevStatus* status = (DevStatus*)(base + kStatusOff);
    // tables (pageable host memory: the copies complete before they return
    // control), then clear the counters and the status word of this call
    if (cudaMemcpyAsync(u.d_origin, org.data(), org.size() * sizeof(int2), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(u.d_prod, prod.data(), prod.size() * sizeof(int4), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemsetAsync(base + kFlagsOff, 0, kStatusOff + sizeof(DevStatus) - kFlagsOff, st) !=
            cudaSuccess)
        return M2S_ERR_CUDA;
    cudaError_t e = dtype == M2S_F64
                        ? run<double>(d, (const double*)b, (double*)x, n_sym_sweeps, base, u, status, st)
                        : run<float>(d, (const float*)b, (float*)x, n_sym_sweeps, base, u, status, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? M2S_ERR_OOM : M2S_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return M2S_ERR_CUDA;
    DevStatus hs;
    if (cudaMemcpy(&hs, status, sizeof(DevStatus), cudaMemcpyDeviceToHost) != cudaSuccess)
        return M2S_ERR_CUDA;
    return hs.err ? (m2s_status)hs.err : M2S_OK;
}
