// Fused step kernel instantiations: D3Q15, storage f32.
#define LBM_LAT D3Q15
#define LBM_STORE ST_F32
#define LBM_FN launch_step_d3q15_f32
#include "lbm_step_inst.cuh"
