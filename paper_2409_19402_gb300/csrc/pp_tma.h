// pp_tma.h -- tensor-map (TMA descriptor) encoding shared by the tensor-core
// translation units.  cuTensorMapEncodeTiled is taken from the driver through
// the runtime's entry-point query, once per process.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace pp {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// A row-major outer x inner FP32 matrix (rows `inner` floats long, contiguous)
// as a 2-D map with box_outer x box_inner boxes, no swizzle, out-of-range
// elements read as zero and clipped on stores.  False when the base is not
// 16-byte aligned, a row is not a multiple of 16 bytes, or the driver refuses.
inline bool encode_rows_2d(CUtensorMap *map, const float *base, int64_t inner, int64_t outer,
                           uint32_t box_inner, uint32_t box_outer, bool l2_promote,
                           bool swizzle128 = false) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || inner % 4 != 0 || inner < 1 ||
      outer < 1)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * sizeof(float)};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
             l2_promote ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// `layers` row-major outer x inner FP32 matrices, one after the other, as a
// 3-D map with box_outer x box_inner x 1 boxes, no swizzle (clipped per layer).
inline bool encode_layers_3d(CUtensorMap *map, const float *base, int64_t inner, int64_t outer,
                             int64_t layers, uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || inner % 4 != 0 || inner < 1 ||
      outer < 1 || layers < 1)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)outer, (cuuint64_t)layers};
  const cuuint64_t strides[2] = {(cuuint64_t)inner * sizeof(float),
                                 (cuuint64_t)(inner * outer) * sizeof(float)};
  const cuuint32_t box[3] = {box_inner, box_outer, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// `layers` matrices of outer x inner FP32 elements, rows `row_stride` floats
// apart and layers `layer_stride` floats apart, as a 3-D map with
// box_outer x box_inner x 1 boxes; out-of-range elements read as zero and are
// clipped on stores.  False when the base is not 16-byte aligned, a stride is
// not a multiple of 16 bytes, or the driver refuses.
inline bool encode_3d(CUtensorMap *map, const float *base, int64_t inner, int64_t outer,
                      int64_t layers, int64_t row_stride, int64_t layer_stride,
                      uint32_t box_inner, uint32_t box_outer, bool l2_promote, bool swizzle128) {
  EncodeTiledFn enc = encode_tiled();
  if (layers == 1) layer_stride = row_stride * outer;   // unused; any valid value
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || inner < 1 || outer < 1 ||
      layers < 1 || row_stride < inner || row_stride % 4 != 0 || layer_stride < 4 ||
      layer_stride % 4 != 0)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)outer, (cuuint64_t)layers};
  const cuuint64_t strides[2] = {(cuuint64_t)row_stride * sizeof(float),
                                 (cuuint64_t)layer_stride * sizeof(float)};
  const cuuint32_t box[3] = {box_inner, box_outer, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
             l2_promote ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace pp
