// Tensor maps for the TMA-staged D2Q9 step (host side). The encoder comes from
// the CUDA driver through the runtime's entry-point query, so the library does
// not link libcuda.
#include <cudaTypedefs.h>

#include "lbm_internal.cuh"

namespace lbm {

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// rank-2 or rank-3 map over [d2][ny][nx] elements of `bytes` each, box (bx, 1[, d2])
static bool encode(PFN_cuTensorMapEncodeTiled_v12000 fn, CUtensorMap* m, const void* base, int rank,
                   CUtensorMapDataType type, int bytes, int nx, int ny, int d2, int bx)
{
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)d2};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * bytes, (cuuint64_t)nx * ny * bytes};
    const cuuint32_t box[3] = {(cuuint32_t)bx, 1u, (cuuint32_t)d2};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(m, type, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_tma_maps(const void* g, const float* phi, const float* ua, int nx, int ny, TmaMaps* out)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn || nx % 256 != 0 || ny < 1) return false;
    bool ok = encode(fn, &out->g, g, 3, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, nx, ny, 9, 256) &&
              encode(fn, &out->gh, g, 3, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, nx, ny, 9, 8) &&
              encode(fn, &out->p, phi, 2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nx, ny, 1, 256) &&
              encode(fn, &out->ph, phi, 2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nx, ny, 1, 4);
    if (ok && ua)
        ok = encode(fn, &out->u, ua, 3, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nx, ny, 2, 256) &&
             encode(fn, &out->uh, ua, 3, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nx, ny, 2, 4);
    else if (ok)
        out->u = out->uh = out->p;   // not read without a velocity field
    return ok;
}

}  // namespace lbm
