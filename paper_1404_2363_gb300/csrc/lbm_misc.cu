// Non-step kernels (initialisation, phi read-out, FP64 sums) and the step
// dispatch over the per-(lattice, storage) translation units.
#include "lbm_device.cuh"

namespace lbm {

cudaError_t launch_step_d2q9_f32(int, bool, LaunchCfg, const StepArgs&, cudaStream_t);
cudaError_t launch_step_d2q9_f16(int, bool, LaunchCfg, const StepArgs&, cudaStream_t);
cudaError_t launch_step_d2q9_bf16(int, bool, LaunchCfg, const StepArgs&, cudaStream_t);
cudaError_t launch_step_d3q15_f32(int, bool, LaunchCfg, const StepArgs&, cudaStream_t);
cudaError_t launch_step_d3q15_f16(int, bool, LaunchCfg, const StepArgs&, cudaStream_t);
cudaError_t launch_step_d3q15_bf16(int, bool, LaunchCfg, const StepArgs&, cudaStream_t);

cudaError_t launch_step(int q, int store, int ukind, bool walls, LaunchCfg cfg, const StepArgs& a,
                        cudaStream_t st)
{
    if (q == 9) {
        if (store == ST_F16) return launch_step_d2q9_f16(ukind, walls, cfg, a, st);
        if (store == ST_BF16) return launch_step_d2q9_bf16(ukind, walls, cfg, a, st);
        return launch_step_d2q9_f32(ukind, walls, cfg, a, st);
    }
    if (store == ST_F16) return launch_step_d3q15_f16(ukind, walls, cfg, a, st);
    if (store == ST_BF16) return launch_step_d3q15_bf16(ukind, walls, cfg, a, st);
    return launch_step_d3q15_f32(ukind, walls, cfg, a, st);
}

__global__ void __launch_bounds__(256) k_sum2(const double* __restrict__ partials, int n,
                                              double* __restrict__ out)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

static int flat_blocks(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152LL * 16) b = 152LL * 16;
    return (int)(b < 1 ? 1 : b);
}

template <class L, int STORE>
static cudaError_t init_u(int uk, const float* phi0, const StepArgs& a, cudaStream_t st)
{
    const int nb = flat_blocks(a.ncell);
    switch (uk) {
        case U_FIELD: k_init<L, STORE, U_FIELD><<<nb, 256, 0, st>>>(a, phi0); break;
        case U_ROW: k_init<L, STORE, U_ROW><<<nb, 256, 0, st>>>(a, phi0); break;
        default: k_init<L, STORE, U_NONE><<<nb, 256, 0, st>>>(a, phi0); break;
    }
    return cudaGetLastError();
}

template <class L>
static cudaError_t init_s(int store, int uk, const float* phi0, const StepArgs& a, cudaStream_t st)
{
    switch (store) {
        case ST_F16: return init_u<L, ST_F16>(uk, phi0, a, st);
        case ST_BF16: return init_u<L, ST_BF16>(uk, phi0, a, st);
        default: return init_u<L, ST_F32>(uk, phi0, a, st);
    }
}

cudaError_t launch_init(int q, int store, int ukind, const float* phi0, const StepArgs& a,
                        cudaStream_t st)
{
    if (q == 9) return init_s<D2Q9>(store, ukind, phi0, a, st);
    return init_s<D3Q15>(store, ukind, phi0, a, st);
}

template <class L>
static cudaError_t phi_s(int store, const StepArgs& a, float* out, cudaStream_t st)
{
    const int nb = flat_blocks(a.ncell);
    switch (store) {
        case ST_F16: k_phi<L, ST_F16><<<nb, 256, 0, st>>>(a, out); break;
        case ST_BF16: k_phi<L, ST_BF16><<<nb, 256, 0, st>>>(a, out); break;
        default: k_phi<L, ST_F32><<<nb, 256, 0, st>>>(a, out); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_phi(int q, int store, const StepArgs& a, float* phi_out, cudaStream_t st)
{
    if (q == 9) return phi_s<D2Q9>(store, a, phi_out, st);
    return phi_s<D3Q15>(store, a, phi_out, st);
}

template <class L>
static void sum1_s(int store, const StepArgs& a, double* partials, int nb, cudaStream_t st)
{
    switch (store) {
        case ST_F16: k_sum1<L, ST_F16><<<nb, 256, 0, st>>>(a, partials); break;
        case ST_BF16: k_sum1<L, ST_BF16><<<nb, 256, 0, st>>>(a, partials); break;
        default: k_sum1<L, ST_F32><<<nb, 256, 0, st>>>(a, partials); break;
    }
}

cudaError_t launch_sum(int q, int store, const StepArgs& a, double* partials, int nblocks,
                       double* out_dev, cudaStream_t st)
{
    if (q == 9) sum1_s<D2Q9>(store, a, partials, nblocks, st);
    else sum1_s<D3Q15>(store, a, partials, nblocks, st);
    k_sum2<<<1, 256, 0, st>>>(partials, nblocks, out_dev);
    return cudaGetLastError();
}

}  // namespace lbm
