// Host-side encoding of the tensor maps of the staged fused kernels (the
// state as a rank-4 tensor {x, y, z, coefficient row}; see tma_ptx.cuh).
// The driver's encoder is looked up once through the runtime, so the library
// does not link the driver library itself.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "tma_ptx.cuh"

namespace hermite {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

}  // namespace

bool encode_state_map(CUtensorMap *map, const void *base, int elem_bytes, int nx, int ny, int nz, int ncoef,
                      int box_x, int box_y) {
  if (elem_bytes != 4 && elem_bytes != 8) return false;
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || ((size_t)nx * elem_bytes) % 16 != 0) return false;
  if (box_x < 1 || box_x > 256 || (box_x * elem_bytes) % 16 != 0 || box_y < 1 || box_y > 256 || ncoef < 1 ||
      ncoef > 256 || box_x > nx || box_y > ny)
    return false;
  const EncodeTiledFn fn = encoder();
  if (!fn) return false;
  const cuuint64_t eb = (cuuint64_t)elem_bytes;
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)ncoef};
  const cuuint64_t strides[3] = {dims[0] * eb, dims[0] * dims[1] * eb, dims[0] * dims[1] * dims[2] * eb};
  const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1u, (cuuint32_t)ncoef};
  const cuuint32_t estride[4] = {1u, 1u, 1u, 1u};
  const CUresult r =
      fn(map, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
         const_cast<void *>(base), dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace hermite
