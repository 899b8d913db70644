// Fused step kernel instantiations: D2Q9, storage f16.
#define LBM_LAT D2Q9
#define LBM_STORE ST_F16
#define LBM_FN launch_step_d2q9_f16
#include "lbm_step_inst.cuh"
