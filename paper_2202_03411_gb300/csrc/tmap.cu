// tmap.cu -- host-side encoding of the TMA tensor maps the tensor-core
// kernels load their 16-bit operand tiles with (the driver's
// cuTensorMapEncodeTiled, looked up once through the runtime).
#include "internal.cuh"

#include <cstring>

namespace scm {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

bool encode_tmap_3d_16bit(CUtensorMap *map, void *base, const uint64_t dims[3], const uint64_t strides[2],
                          const uint32_t box[3], bool bf16, std::string *why, int swizzle_bytes) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult qr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                                         &qr);
        if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !ptr) {
            *why = "cuTensorMapEncodeTiled is not available from the driver";
            return false;
        }
        fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    std::memset(map, 0, sizeof(CUtensorMap));
    cuuint64_t d[3] = {dims[0], dims[1], dims[2]};
    cuuint64_t st[2] = {strides[0], strides[1]};
    cuuint32_t bx[3] = {box[0], box[1], box[2]};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapSwizzle sw = swizzle_bytes == 32   ? CU_TENSOR_MAP_SWIZZLE_32B
                                  : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                        : CU_TENSOR_MAP_SWIZZLE_128B;
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, d, st, bx,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
        return false;
    }
    return true;
}

}  // namespace scm
