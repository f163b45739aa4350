// The subdomain "box" of the Vanka smoothers (Sec. 3), shared by the
// single-problem and batched kernels.
//
// Subdomain i = pressure DoF p_i + the free velocity DoFs of the cells around
// vertex i.  On a tensor grid these are the positions of a fixed box: Q2 nodes
// J = 2i - 2 + a, a in [0,5)^d, every component, then p_i; box position
// k = d (a0 + 5 a1 + 25 a2) + c, pressure last.  Owned (restricted, Eq. 13)
// rows: nodes a in {2,3}^d (J = 2i + delta) and p_i.
#pragma once

#include "common.cuh"

namespace rav {

template <int D>
struct BoxT {
  static constexpr int NV = D == 2 ? 25 : 125;      // box nodes
  static constexpr int NC = D * NV + 1;             // box positions
  static constexpr int NON = 1 << D;                // owned nodes
  static constexpr int NR = D * NON + 1;            // owned rows
  static constexpr int RB = D == 2 ? 9 : 5;         // owned rows per thread in the RAV apply
  static constexpr int NCH = NR / RB;               // threads per subdomain in the RAV apply
  static constexpr int NF = NON * NV + D * NV + 1;  // factored storage per subdomain
};

// Vertex tuple of subdomain p.
__device__ __forceinline__ void vertex_of(const Geo& g, int64_t p, int* v) {
  for (int a = 0; a < g.dim; ++a) { v[a] = (int)(p % (g.N + 1)); p /= (g.N + 1); }
}
// Same for a compile-time dimension, in 32-bit arithmetic (vertex counts stay
// below 2^31), so that v stays in registers.
template <int D>
__device__ __forceinline__ void vertex_of_t(const Geo& g, int64_t p, int* v) {
  unsigned q = (unsigned)p;
  const unsigned m = (unsigned)g.N + 1;
#pragma unroll
  for (int a = 0; a < D; ++a) { v[a] = (int)(q % m); q /= m; }
}
// Box node a (per-axis offsets) of subdomain at vertex v is valid iff
// 1 <= 2v - 2 + a <= 2N - 1 on every axis (inside, not on the boundary).
__device__ __forceinline__ bool box_node_valid(const Geo& g, const int* v, const int* a) {
  bool ok = true;
  for (int d = 0; d < g.dim; ++d) {
    const int J = 2 * v[d] - 2 + a[d];
    ok &= (J >= 1) & (J <= 2 * g.N - 1);
  }
  return ok;
}
__device__ __forceinline__ void box_tuple(int D, int m, int* a) {
  a[0] = m % 5;
  a[1] = (m / 5) % 5;
  a[2] = D == 3 ? m / 25 : 0;
}

}  // namespace rav
