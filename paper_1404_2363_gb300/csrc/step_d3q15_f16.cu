// Fused step kernel instantiations: D3Q15, storage f16.
#define LBM_LAT D3Q15
#define LBM_STORE ST_F16
#define LBM_FN launch_step_d3q15_f16
#include "lbm_step_inst.cuh"
