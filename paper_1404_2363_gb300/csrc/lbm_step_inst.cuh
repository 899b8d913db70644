// Launch dispatch for one (lattice, storage) pair of the fused step kernel.
// Each step_*.cu translation unit includes this with LBM_LAT / LBM_STORE /
// LBM_FN defined, so the template instantiations compile in parallel.
#include "lbm_device.cuh"
#include "lbm_pair.cuh"
#include "lbm_pair_d3q15.cuh"
#include "lbm_tma_d2q9.cuh"
#include "lbm_zwalk_d3q15.cuh"

namespace lbm {

template <class L, int STORE, int UK, bool WALLS>
static cudaError_t step_vec(LaunchCfg cfg, const StepArgs& a, cudaStream_t st)
{
    if (a.bcx_lo != BC_PERIODIC || a.bcz_lo != BC_PERIODIC) {
        // walls on the x or z faces: the general one-node kernel, whatever the launch shape
        dim3 grid((unsigned)((a.nx + 255) / 256), (unsigned)a.ny, (unsigned)a.nz);
        if ((long long)(L::Q + 3) * a.ncell < (1LL << 31)) k_step_box<L, STORE, UK, int><<<grid, 256, 0, st>>>(a);
        else k_step_box<L, STORE, UK, long long><<<grid, 256, 0, st>>>(a);
        return cudaGetLastError();
    }
    if constexpr (L::Q == 9) {
        if (cfg.vec == 6 && quad_ok(a, UK)) {
            // node-quad variant: 128-bit / 64-bit vector loads and stores, four nodes per thread
            const int per = 4 * cfg.block;
            dim3 grid((unsigned)((a.nx + per - 1) / per), (unsigned)a.ny, 1);
            k_step_quad_d2q9<STORE, UK, WALLS><<<grid, cfg.block, 0, st>>>(a);
            return cudaGetLastError();
        }
    }
    if constexpr (L::Q == 15 && STORE != ST_F32) {
        // phi, the velocity factors and the offsets staged in shared memory along a walk in z
        if (cfg.vec == 9 && cfg.block == 256 && zw_ok(a, UK, 8)) return launch_zw_d3q15<STORE, UK, WALLS, 8>(a, st);
        if (cfg.vec == 9 && cfg.block == 128 && zw_ok(a, UK, 4)) return launch_zw_d3q15<STORE, UK, WALLS, 4>(a, st);
        if (cfg.vec == 5 && pair_ok(a, UK, L::Q)) {
            // node-pair variant (paired FP32 arithmetic, two adjacent nodes per thread)
            const int per = 2 * cfg.block;
            dim3 grid((unsigned)((a.nx + per - 1) / per), (unsigned)a.ny, (unsigned)a.nz);
            k_step_pair_d3q15<STORE, UK, WALLS><<<grid, cfg.block, 0, st>>>(a);
            return cudaGetLastError();
        }
    }
    if constexpr (L::Q == 9 && STORE != ST_F32) {
        // TMA-staged rows: two rows per iteration and six stages, or one row and four
        if (cfg.vec == 7 && tma_ok(a, UK)) return launch_tma_d2q9<STORE, UK, WALLS, 2, 6>(a, st);
        if (cfg.vec == 8 && tma_ok(a, UK)) return launch_tma_d2q9<STORE, UK, WALLS, 1, 4>(a, st);
        if (cfg.vec == 5 && a.nz == 1 && pair_ok(a, UK, L::Q)) {
            // node-pair variant (paired FP32 arithmetic, two adjacent nodes per thread)
            const int per = 2 * cfg.block;
            dim3 grid((unsigned)((a.nx + per - 1) / per), (unsigned)a.ny, 1);
            k_step_pair_d2q9<STORE, UK, WALLS><<<grid, cfg.block, 0, st>>>(a);
            return cudaGetLastError();
        }
    }
    const int vec = cfg.vec == 2 ? 2 : 1;
    const int per = cfg.block * vec;
    dim3 grid((unsigned)((a.nx + per - 1) / per), (unsigned)a.ny, (unsigned)a.nz);
    dim3 block((unsigned)cfg.block);
    // 32-bit offsets when every plane and velocity offset fits
    const bool idx32 = (long long)(L::Q + 3) * a.ncell < (1LL << 31);
    if (idx32) {
        if (vec == 2) k_step<L, STORE, UK, WALLS, 2, int><<<grid, block, 0, st>>>(a);
        else k_step<L, STORE, UK, WALLS, 1, int><<<grid, block, 0, st>>>(a);
    } else {
        if (vec == 2) k_step<L, STORE, UK, WALLS, 2, long long><<<grid, block, 0, st>>>(a);
        else k_step<L, STORE, UK, WALLS, 1, long long><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <class L, int STORE, int UK>
static cudaError_t step_w(bool walls, LaunchCfg cfg, const StepArgs& a, cudaStream_t st)
{
    return walls ? step_vec<L, STORE, UK, true>(cfg, a, st) : step_vec<L, STORE, UK, false>(cfg, a, st);
}

cudaError_t LBM_FN(int uk, bool walls, LaunchCfg cfg, const StepArgs& a, cudaStream_t st)
{
    switch (uk) {
        case U_FIELD: return step_w<LBM_LAT, LBM_STORE, U_FIELD>(walls, cfg, a, st);
        case U_ROW: return step_w<LBM_LAT, LBM_STORE, U_ROW>(walls, cfg, a, st);
        default: return step_w<LBM_LAT, LBM_STORE, U_NONE>(walls, cfg, a, st);
    }
}

}  // namespace lbm
