// render.cuh -- the sprite renderer's pixel rule, shared by the frame renderer
// and the fused conv1 producer (which renders its operand tiles on the fly).
#pragma once

#include "common.cuh"

namespace bcts {

// Sprite masks (4x4, bit r*4+c) and palette of objects 0..3, packed:
// agent = full block 240, reward = diamond 192, hazards = X 128 and ring 64.
constexpr uint64_t kSprites = 0xF99F96696FF6FFFFull;
constexpr uint32_t kPalette = 0x4080C0F0u;

// Object cells of one history slot from the 16 bytes pos[h][0..3][x, y].
__device__ __forceinline__ void unpack_slot(const uint4 P, int ox[4], int oy[4]) {
  const uint32_t pw[4] = {P.x, P.y, P.z, P.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ox[k] = int(int16_t(pw[k] & 0xFFFFu));
    oy[k] = int(int16_t(pw[k] >> 16));
  }
}

// The 4 pixels (little-endian bytes) of cell column cx in pixel row y: objects
// are painted in index order, a later object's set sprite bits overwrite.
__device__ __forceinline__ uint32_t render_word(const int ox[4], const int oy[4], int cx, int y) {
  const int cy = y >> 2, sr = y & 3;
  uint32_t v = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (ox[k] == cx && oy[k] == cy) {
      const uint32_t bits = uint32_t(kSprites >> (16 * k + 4 * sr)) & 0xFu;
      const uint32_t bytemask = ((bits * 0x00204081u) & 0x01010101u) * 0xFFu;
      const uint32_t pal = ((kPalette >> (8 * k)) & 0xFFu) * 0x01010101u;
      v = (v & ~bytemask) | (pal & bytemask);
    }
  }
  return v;
}

}  // namespace bcts
