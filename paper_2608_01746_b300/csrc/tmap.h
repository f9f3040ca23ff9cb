// Host-side encoding of TMA tensor maps (cuTensorMapEncodeTiled, fetched from the driver once).
#pragma once

#include <cuda.h>
#include <stddef.h>
#include <stdint.h>

namespace pm {

// Row-major 2-D tensor [outer][inner] of `esize`-byte elements at `addr` (16-byte aligned,
// inner * esize a multiple of 16), box {box_in, box_out} elements, swizzle `sw`.  Returns
// PTYCHO_OK or PTYCHO_ECUDA (message in the last-error slot).
int encode_2d(CUtensorMap *m, void *addr, CUtensorMapDataType dt, size_t esize, uint64_t inner, uint64_t outer,
              uint32_t box_in, uint32_t box_out, CUtensorMapSwizzle sw);

}  // namespace pm
