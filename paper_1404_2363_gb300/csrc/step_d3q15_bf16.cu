// Fused step kernel instantiations: D3Q15, storage bf16.
#define LBM_LAT D3Q15
#define LBM_STORE ST_BF16
#define LBM_FN launch_step_d3q15_bf16
#include "lbm_step_inst.cuh"
