// Host-side encoding of TMA tensor maps for padded frames (driver entry point looked
// up through the runtime, so the library does not link libcuda directly).
#include <cudaTypedefs.h>

#include "osbf_internal.h"

namespace osbf {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// A 3-D map over P frames of FH rows x FW elements (row pitch `pitch` elements).  Reads
// outside [0, FW) x [0, FH) return zeros -- the appendix's "zero outside the padded frame"
// (for selection maps, U8: window index 0, "no window").
bool encode_frame_map(CUtensorMap *map, Storage st, const void *base, int FW, int FH, int P, int pitch, int box_w,
                      int box_h) {
    auto fn = encode_fn();
    if (!fn) return false;
    CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    int es = 4;
    if (st == Storage::F16) {
        dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
        es = 2;
    } else if (st == Storage::BF16) {
        dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        es = 2;
    } else if (st == Storage::U8) {
        dt = CU_TENSOR_MAP_DATA_TYPE_UINT8;
        es = 1;
    }
    cuuint64_t dims[3] = {(cuuint64_t)FW, (cuuint64_t)FH, (cuuint64_t)P};
    cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)pitch * es * FH};
    cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_store_map(CUtensorMap *map, void *base, int W, int H, int P, int pitch) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)P};
    cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * 4 * H};
    cuuint32_t box[3] = {32, 32, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace osbf
