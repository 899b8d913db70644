// Fused step kernel instantiations: D2Q9, storage f32.
#define LBM_LAT D2Q9
#define LBM_STORE ST_F32
#define LBM_FN launch_step_d2q9_f32
#include "lbm_step_inst.cuh"
