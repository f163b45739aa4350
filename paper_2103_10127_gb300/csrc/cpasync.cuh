// Asynchronous global -> shared copies (cp.async, sm_80 and later) and the
// chunk decoders shared by the streamed subdomain applies (staged.cu,
// stream.cu).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

namespace rav {

__device__ __forceinline__ uint32_t st_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Asynchronous copy of BYTES (4, 8 or a multiple of 16) from global to shared
// memory; both addresses aligned to min(BYTES, 16).
template <int BYTES>
__device__ __forceinline__ void st_copy(void* dst, const void* src) {
  if constexpr (BYTES % 16 == 0) {
#pragma unroll
    for (int i = 0; i < BYTES; i += 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(st_smem((char*)dst + i)),
                   "l"((const char*)src + i)
                   : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(st_smem(dst)), "l"(src), "n"(BYTES) : "memory");
  }
}
// cp.async of 4, 8 or 16 bytes, zero-filled when !valid (src is not read then).
__device__ __forceinline__ void st_copy4z(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(st_smem(dst)), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void st_copy8z(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(st_smem(dst)), "l"(src), "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void st_copy16z(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(st_smem(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void st_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Waits until at most N of this thread's copy groups are pending.
template <int N>
__device__ __forceinline__ void st_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Widens NW 32-bit words of stored values of type T to fp32 (bf16 pairs: the
// lower address is the low half of the word).
template <typename T, int NW>
__device__ __forceinline__ void widen_words(const unsigned* w, float* out) {
  if constexpr (std::is_same<T, float>::value) {
#pragma unroll
    for (int i = 0; i < NW; ++i) out[i] = __uint_as_float(w[i]);
  } else {
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      out[2 * i] = __uint_as_float(w[i] << 16);
      out[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
}

// NVAL consecutive stored values (one chunk of NVAL * sizeof(T) bytes, aligned
// to that size, 4 to 32 bytes) from global memory, widened to fp32; read once
// per pass, hence the evict-first loads.
template <typename T, int NVAL>
__device__ __forceinline__ void ld_chunk(const T* __restrict__ p, float* out) {
  constexpr int BYTES = NVAL * (int)sizeof(T);
  constexpr int NW = BYTES / 4;
  unsigned w[NW];
  if constexpr (BYTES == 4) {
    w[0] = __ldcs(reinterpret_cast<const unsigned*>(p));
  } else if constexpr (BYTES == 8) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
    w[0] = v.x;
    w[1] = v.y;
  } else {
#pragma unroll
    for (int i = 0; i < NW; i += 4) {
      const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p) + i / 4);
      w[i] = v.x;
      w[i + 1] = v.y;
      w[i + 2] = v.z;
      w[i + 3] = v.w;
    }
  }
  widen_words<T, NW>(w, out);
}

// The same for a chunk already in shared memory.
template <typename T, int NVAL>
__device__ __forceinline__ void sm_chunk(const T* p, float* out) {
  constexpr int NW = NVAL * (int)sizeof(T) / 4;
  unsigned w[NW];
  if constexpr (NW == 1) {
    w[0] = *reinterpret_cast<const unsigned*>(p);
  } else if constexpr (NW == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    w[0] = v.x;
    w[1] = v.y;
  } else {
#pragma unroll
    for (int i = 0; i < NW; i += 4) {
      const uint4 v = reinterpret_cast<const uint4*>(p)[i / 4];
      w[i] = v.x;
      w[i + 1] = v.y;
      w[i + 2] = v.z;
      w[i + 3] = v.w;
    }
  }
  widen_words<T, NW>(w, out);
}

// BYTES of one chunk as 32-bit words, read once (evict-first).
template <int BYTES>
struct RawChunk {
  unsigned w[BYTES / 4];
};
template <int BYTES>
__device__ __forceinline__ RawChunk<BYTES> ld_raw(const void* p) {
  RawChunk<BYTES> r;
  if constexpr (BYTES == 4) {
    r.w[0] = __ldcs(reinterpret_cast<const unsigned*>(p));
  } else if constexpr (BYTES == 8) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
    r.w[0] = v.x;
    r.w[1] = v.y;
  } else {
#pragma unroll
    for (int i = 0; i < BYTES / 16; ++i) {
      const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p) + i);
      r.w[4 * i] = v.x;
      r.w[4 * i + 1] = v.y;
      r.w[4 * i + 2] = v.z;
      r.w[4 * i + 3] = v.w;
    }
  }
  return r;
}

// One staged residual node: d fp32 components (3-D padded to 16 bytes).
template <int D>
struct NodeT;
template <>
struct NodeT<2> {
  using type = float2;
};
template <>
struct NodeT<3> {
  using type = float4;
};

}  // namespace rav
