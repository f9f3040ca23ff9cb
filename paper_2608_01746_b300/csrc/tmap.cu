// Host-side encoding of TMA tensor maps (see tmap.h).
#include <mutex>

#include "common.cuh"
#include "tmap.h"

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_enc_mu;
EncodeTiledFn g_enc = nullptr;

int tensor_map_encoder(EncodeTiledFn *fn) {
    std::lock_guard<std::mutex> lk(g_enc_mu);
    if (!g_enc) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        PM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p)
            return pm::fail(PTYCHO_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
        g_enc = (EncodeTiledFn)p;
    }
    *fn = g_enc;
    return PTYCHO_OK;
}

}  // namespace

namespace pm {

int encode_2d(CUtensorMap *m, void *addr, CUtensorMapDataType dt, size_t esize, uint64_t inner, uint64_t outer,
              uint32_t box_in, uint32_t box_out, CUtensorMapSwizzle sw) {
    EncodeTiledFn enc;
    int rc = tensor_map_encoder(&enc);
    if (rc) return rc;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * esize};
    const cuuint32_t box[2] = {box_in, box_out};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, dt, 2, addr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return pm::fail(PTYCHO_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PTYCHO_OK;
}

}  // namespace pm
