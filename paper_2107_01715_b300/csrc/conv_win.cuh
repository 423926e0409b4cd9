// conv_win.cuh -- geometry of the shared-memory window form of conv2 / conv3 and
// the tensor map that loads a window, shared by the window kernels (conv_win.cu)
// and the tap-pair kernel (conv_pair.cu).
//
// Stride-1 form.  Number the rows (pixels) of an NHWC map r = node*H*W + y*W + x.
// Output (y, x) of a stride-1 K x K convolution reads, at filter tap (ky, kx),
// input row r + ky*W + kx: the same shift for every output row once the output
// grid is padded to the input's width and height.  conv3 (3x3 / 1 on [9][9][64])
// has this form as it is; conv2 (4x4 / 2 on [20][20][32]) has it on the
// space-to-depth view of its input: [10][10] super-pixels of 2 x 2 pixels and
// 128 channels (dy, dx, c), a 2 x 2 stride-1 filter.  In the NHWC map the 64
// channels (dx, c) of super-pixel row dy are 64 contiguous elements, so a 4D
// tiled TMA box (channels, x2, dy, node*10 + y2) reads the view as stored: window
// slab dy holds rows (y2, x2), and its weights are 64 consecutive K of the
// (ky, kx, c) order.
#pragma once

#include <stdint.h>

#include "../../include/bcts.h"
#include "tma_host.cuh"

namespace bcts {
namespace tc {

template <int LAYER>
struct WinGeo;
template <>
struct WinGeo<2> {  // space-to-depth view of [20][20][32]: [10][10] x (dy, dx, c)
  static constexpr int PW = 10, PP = 100;  // padded grid width, padded rows per node
  static constexpr int OW = 9, P = 81;     // output side, output pixels per node
  static constexpr int TW = 2, NTAP = 4;   // filter side and taps over super-pixels
  static constexpr int NSLAB = 2;          // window slabs per row (dy)
  static constexpr int LINES = 15;         // window lines of PW rows loaded per tile
  static constexpr int WROWS = LINES * PW; // 150 >= 9 (tile start in its line) + 128 + 11 (largest shift)
  __host__ __device__ static constexpr int wx(int tap, int slab) {  // first K of (tap, slab) in (ky, kx, c)
    return ((2 * (tap / 2) + slab) * 4 + 2 * (tap % 2)) * 32;
  }
};
template <>
struct WinGeo<3> {  // [9][9][64]
  static constexpr int PW = 9, PP = 81;
  static constexpr int OW = 7, P = 49;
  static constexpr int TW = 3, NTAP = 9;
  static constexpr int NSLAB = 1;
  static constexpr int WROWS = 148;        // 128 + 20 (largest shift)
  __host__ __device__ static constexpr int wx(int tap, int) { return tap * 64; }
};

// The input window map of n nodes, bf16 (fp8 = false) or one-byte E4M3 elements.
// conv2: 4D view (channels (dx, c), x2, dy, node*10 + y2) of the NHWC
// [n][20][20][32] map, box = 15 lines of 10 super-pixels of one dy.  conv3:
// [n*81][64] rows, box = 148 rows.  Rows past the end read as zeros.
template <int LAYER>
inline int encode_window_map(CUtensorMap *m, const void *base, int64_t n, bool fp8) {
  using G = WinGeo<LAYER>;
  const Encoders &e = encoders();
  if (!e.tiled) return BCTS_ECUDA;
  const int eb = fp8 ? 1 : 2;
  const CUtensorMapDataType dt = fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUresult r;
  if constexpr (LAYER == 2) {
    const cuuint64_t dims[4] = {64, 10, 2, cuuint64_t(n) * 10};
    const cuuint64_t strides[3] = {cuuint64_t(64 * eb), cuuint64_t(640 * eb), cuuint64_t(1280 * eb)};
    const cuuint32_t box[4] = {64, 10, 1, cuuint32_t(G::LINES)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    r = e.tiled(m, dt, 4, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                swizzle_for(64 * eb), CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const cuuint64_t dims[2] = {64, cuuint64_t(n) * G::PP};
    const cuuint64_t strides[1] = {cuuint64_t(64 * eb)};
    const cuuint32_t box[2] = {64, cuuint32_t(G::WROWS)};
    const cuuint32_t estr[2] = {1, 1};
    r = e.tiled(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                swizzle_for(64 * eb), CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return r == CUDA_SUCCESS ? BCTS_OK : BCTS_ECUDA;
}

}  // namespace tc
}  // namespace bcts
