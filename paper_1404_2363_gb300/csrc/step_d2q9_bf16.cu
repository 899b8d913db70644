// Fused step kernel instantiations: D2Q9, storage bf16.
#define LBM_LAT D2Q9
#define LBM_STORE ST_BF16
#define LBM_FN launch_step_d2q9_bf16
#include "lbm_step_inst.cuh"
