// Allocation-free FP64 sum of phi over a raw solver state.
//
// Some callers cannot allocate device memory at the point where they need a
// conservation check: code that runs while a stream is being captured into a
// CUDA graph, real-time loops that forbid allocator calls, or hosts that hand
// the library a fixed memory budget. lbm_cde_sum_state_noalloc serves them: it
// is the two-pass deterministic FP64 reduction of lbm_cde_sum_phi, but its
// per-block partial sums live in a file-scope __device__ array instead of a
// buffer the handle allocates, and it takes the state by pointer instead of a
// handle.
//
// Limits and sharing:
//   * the scratch holds LBM_NOALLOC_MAX_PARTIALS doubles (128 KiB per GPU, kept
//     for the life of the process on every GPU that loads the library); each
//     partial covers LBM_NOALLOC_CELLS_PER_BLOCK cells, so a state may have at
//     most LBM_NOALLOC_MAX_CELLS cells; larger states are rejected;
//   * every call overwrites the partials it uses and writes its result (no
//     accumulation), so nothing has to be zeroed between calls;
//   * all calls on a GPU share the one array: calls whose kernels overlap on
//     the GPU (different streams without ordering) race and give wrong sums.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/lbm_cde.h"
#include "lbm_device.cuh"

namespace {

constexpr long long kMaxPartials = LBM_NOALLOC_MAX_PARTIALS;
constexpr long long kCellsPerBlock = LBM_NOALLOC_CELLS_PER_BLOCK;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_noalloc_partials[kMaxPartials];

template <class L, int STORE>
__global__ void __launch_bounds__(kThreads) k_noalloc_sum1(const void* state, long long ncell,
                                                          double* __restrict__ partials)
{
    using T = typename lbm::StT<STORE>::T;
    const T* src = static_cast<const T*>(state);
    // the 16-bit forms keep phi as an FP32 plane after the q storage planes
    const float* phi = reinterpret_cast<const float*>(src + (long long)L::Q * ncell);
    const long long c0 = (long long)blockIdx.x * kCellsPerBlock;
    const long long c1 = c0 + kCellsPerBlock < ncell ? c0 + kCellsPerBlock : ncell;
    double acc = 0.0;
    for (long long c = c0 + threadIdx.x; c < c1; c += kThreads) {
        if (STORE != lbm::ST_F32) {
            acc += (double)phi[c];
        } else {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) s += (double)lbm::ldg_f(src + (long long)i * ncell + c);
            acc += s;
        }
    }
    __shared__ double red[kThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kThreads) k_noalloc_sum2(const double* __restrict__ partials, int n,
                                                          double* __restrict__ out)
{
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) acc += partials[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Device address of g_noalloc_partials, resolved once per device with that
// device current. Host code must not pass the symbol itself to a kernel: on
// the host it names a shadow variable, not device memory. The cached address
// belongs to the device's primary context of the moment; a device reset in
// this process would move the array, and calls after one are unsupported.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

cudaError_t partials_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

template <class L>
cudaError_t launch(int storage, const void* state, long long ncell, double* partials, int nb,
                   cudaStream_t st)
{
    switch (storage) {
        case LBM_STORE_F16_NEQ:
            k_noalloc_sum1<L, lbm::ST_F16><<<nb, kThreads, 0, st>>>(state, ncell, partials);
            break;
        case LBM_STORE_BF16_NEQ:
            k_noalloc_sum1<L, lbm::ST_BF16><<<nb, kThreads, 0, st>>>(state, ncell, partials);
            break;
        default:
            k_noalloc_sum1<L, lbm::ST_F32><<<nb, kThreads, 0, st>>>(state, ncell, partials);
            break;
    }
    return cudaGetLastError();
}

thread_local char g_err[256];

}  // namespace

extern "C" lbm_status lbm_cde_sum_state_noalloc(const void* state_dev, int32_t lattice, int32_t storage,
                                                int64_t ncell, double* sum_dev, void* stream)
{
    g_err[0] = 0;
    if (!state_dev || !sum_dev) {
        snprintf(g_err, sizeof(g_err), "state_dev and sum_dev must be device pointers");
        return LBM_E_ARG;
    }
    if ((lattice != LBM_D2Q9 && lattice != LBM_D3Q15) || storage < LBM_STORE_F32 ||
        storage > LBM_STORE_BF16_NEQ || ncell < 1) {
        snprintf(g_err, sizeof(g_err), "bad lattice, storage or ncell");
        return LBM_E_ARG;
    }
    const int q = lattice;
    if ((reinterpret_cast<uintptr_t>(state_dev) % 4) != 0 ||
        (storage != LBM_STORE_F32 && ((long long)q * ncell) % 2 != 0)) {
        snprintf(g_err, sizeof(g_err), "state_dev or its phi plane is not 4-byte aligned");
        return LBM_E_ARG;
    }
    if (ncell > (int64_t)LBM_NOALLOC_MAX_CELLS) {
        snprintf(g_err, sizeof(g_err),
                 "ncell = %lld exceeds the allocation-free limit of %lld cells (%lld partials of %lld cells)",
                 (long long)ncell, (long long)LBM_NOALLOC_MAX_CELLS, kMaxPartials, kCellsPerBlock);
        return LBM_E_ARG;
    }
    double* partials = nullptr;
    cudaError_t e = partials_for_current_device(&partials);
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof(g_err), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return LBM_E_CUDA;
    }
    const int nb = (int)((ncell + kCellsPerBlock - 1) / kCellsPerBlock);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = lattice == LBM_D2Q9 ? launch<lbm::D2Q9>(storage, state_dev, ncell, partials, nb, st)
                            : launch<lbm::D3Q15>(storage, state_dev, ncell, partials, nb, st);
    if (e == cudaSuccess) {
        k_noalloc_sum2<<<1, kThreads, 0, st>>>(partials, nb, sum_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof(g_err), "launch: %s", cudaGetErrorString(e));
        return LBM_E_CUDA;
    }
    return LBM_OK;
}

extern "C" const char* lbm_cde_noalloc_last_error(void) { return g_err; }
