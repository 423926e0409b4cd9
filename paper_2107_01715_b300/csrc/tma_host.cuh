// tma_host.cuh -- host side of the TMA-fed kernels: the tensor-map encoders
// (reached through the runtime's driver entry point, so the library needs no
// link against the driver) and the SM count the persistent grids are sized by.
#pragma once

#include <cuda.h>  // CUtensorMap and its enums
#include <cuda_runtime.h>

namespace bcts {
namespace tc {

using EncodeIm2col = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const int *, const int *, cuuint32_t, cuuint32_t,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct Encoders {
  EncodeIm2col im2col = nullptr;
  EncodeTiled tiled = nullptr;
};

// Resolved once; a member is NULL when the driver does not provide it.
const Encoders &encoders();
// The swizzle mode whose span is `rowb` bytes (32, 64 or 128).
CUtensorMapSwizzle swizzle_for(int rowb);
// SMs of the current device (148 if the query fails).
int num_sms_tma();

}  // namespace tc
}  // namespace bcts
