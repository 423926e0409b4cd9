// tc_ptx.cuh -- inline-PTX wrappers for the tensor-core kernels (tcgen05.mma with
// TMEM accumulators, mbarriers, cp.async and TMA bulk tensor copies) and the
// bounded barrier wait every role of those kernels uses.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace bcts {
namespace tc {

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// Arrive on `bar` (counted in its expected arrivals) once every cp.async this
// thread issued before has landed in shared memory.
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void st_shared16(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// 8 uint8 pixels (two little-endian words) -> 8 bf16.  A pixel b becomes the
// float 2^23 + b by byte permutation, minus 2^23 gives b exactly (integers
// below 256 have at most 8 significant bits, so the bf16 is the top half).
__device__ __forceinline__ uint4 pixels8_to_bf16(uint32_t w0, uint32_t w1) {
  uint32_t o[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const uint32_t w = h < 2 ? w0 : w1;
    const uint32_t j = 2 * (h & 1);
    float2 f = make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u + j)),
                           __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440u + j + 1)));
    f = __fadd2_rn(f, make_float2(-8388608.0f, -8388608.0f));  // both exact
    o[h] = __byte_perm(__float_as_uint(f.x), __float_as_uint(f.y), 0x7632);  // the two upper halves
  }
  return make_uint4(o[0], o[1], o[2], o[3]);
}

// Shared-memory matrix descriptor: K-major tile, 128-byte rows, 128-byte
// swizzle, 8-row groups 1024 bytes apart (the tile base is 1024-byte aligned).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);  // start address
  d |= uint64_t(1) << 16;                  // leading-dimension offset (unused for this layout)
  d |= uint64_t(1024 >> 4) << 32;          // stride between 8-row groups
  d |= uint64_t(1) << 46;                  // descriptor version
  d |= uint64_t(2) << 61;                  // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: bf16 A and B, FP32 accumulator, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

// Instruction descriptor, kind::f8f6f4: E4M3 A and B, FP32 accumulator, K-major,
// M = 128, N = n (K = 32 elements = 32 bytes per instruction).
__host__ __device__ constexpr uint32_t idesc_e4m3(int n) {
  return (1u << 4) | (0u << 7) | (0u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

// 16 uint8 pixels (four little-endian words) -> 16 E4M3 codes (saturating,
// round to nearest; the renderer's palette values are exact).
__device__ __forceinline__ uint4 pixels16_to_e4m3(const uint32_t (&w)[4]) {
  uint32_t o[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float f[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) f[b] = __uint_as_float(__byte_perm(w[h], 0x4B000000u, 0x7440u + b)) - 8388608.0f;
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(f[0], f[1]), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(f[2], f[3]), __NV_SATFINITE, __NV_E4M3);
    o[h] = lo | (hi << 16);
  }
  return make_uint4(o[0], o[1], o[2], o[3]);
}

// Byte offset of 16-byte chunk `ch` of row `r` in a 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t sw128_off(int r, int ch) {
  return uint32_t(r) * 128u + (uint32_t(ch ^ (r & 7)) << 4);
}

constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at the maximum SM clock

// Bounded mbarrier wait.  On time-out: error code into the device error word,
// abort flag for the whole CTA, returns false.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *d_err,
                                         int code, long long limit = kWaitCycles) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  int spins = 0;
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (++spins > 4096) __nanosleep(32);
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      if (d_err) atomicCAS(d_err, 0, code);
      return false;
    }
  }
  return true;
}

// Bounded wait that ignores the abort flag: used at teardown, to let copies and
// MMAs that were issued complete before the CTA releases its shared memory.
__device__ __forceinline__ void wait_bar_drain(uint32_t bar, uint32_t parity, int *d_err) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    __nanosleep(64);
    if (clock64() - t0 > kWaitCycles) {
      if (d_err) atomicCAS(d_err, 0, 5);
      return;
    }
  }
}

// ---- TMA (cp.async.bulk.tensor) ------------------------------------------
// Arrive on `bar` and add `bytes` to the transaction count its phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_prefetch_map(const void *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}
// Tiled 2D load of one box at (x, y) (x innermost, in elements) into shared memory.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// Tiled 4D load of one box at (c0, c1, c2, c3) (c0 innermost, in elements).
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
          dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
// im2col load from a 4D NHWC tensor: pixels traversed from (w, h, n) through the
// map's bounding box (with its traversal strides), each shifted by the filter
// offset (ow, oh); c is the first channel.
__device__ __forceinline__ void tma_load_im2col_4d(uint32_t dst, const void *map, int c, int w, int h, int n,
                                                   uint16_t ow, uint16_t oh, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.im2col.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6], {%7, %8};" ::"r"(dst),
      "l"(map), "r"(c), "r"(w), "r"(h), "r"(n), "r"(bar), "h"(ow), "h"(oh)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with `rowb`-byte rows (32, 64
// or 128) in the matching swizzle mode, 8-row groups 8 * rowb bytes apart; the
// tile base is aligned to 1024 bytes.
__device__ __forceinline__ uint64_t swz_desc(uint32_t saddr, int rowb) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);           // start address
  d |= uint64_t(1) << 16;                           // leading-dimension offset (unused: K fits one row)
  d |= uint64_t((8 * rowb) >> 4) << 32;             // stride between 8-row groups
  d |= uint64_t(1) << 46;                           // descriptor version
  const uint64_t mode = rowb == 128 ? 2 : (rowb == 64 ? 4 : 6);  // 128-, 64- or 32-byte swizzle
  d |= mode << 61;
  return d;
}

}  // namespace tc
}  // namespace bcts
