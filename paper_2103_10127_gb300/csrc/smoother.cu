// Vanka smoothers (Sec. 3): subdomain set-up and application.
//
// Subdomain i = pressure DoF p_i + the free velocity DoFs of the cells around
// vertex i.  On a tensor grid its DoFs are the positions of a fixed "box":
// Q2 nodes J = 2i - 2 + a, a in [0,5)^d, all components, then p_i; box
// position k = d (a0 + 5 a1 + 25 a2) + c, pressure last (n_box = 5^d d + 1).
// A position whose node lies outside the domain or on the boundary is not in
// the subdomain; it keeps a zero row and column, so every subdomain is handled
// with the same padded shape.  Ascending box position = ascending DoF index,
// so the compact subdomain list of the paper is the box filtered by validity.
//
// Local inverse.  The operator is L_i = [A_i b; b^T 0] with one pressure and
// A_i = I_d (x) K_i (the gradient form of Eq. 7 does not couple velocity
// components).  With w = A_i^{-1} b and the scalar Schur complement
// s = -b^T w the block inverse is
//     L_i^{-1} = [A_i^{-1} + w w^T / s,  -w / s;  -w^T / s,  1 / s],
// so one fp64 Cholesky factorisation of K_i (5^d nodes) replaces the LU of the
// full (5^d d + 1)-square system: the paper's L_i^{-1} (Eq. 11) computed
// exactly, at 1/d^3 of the cost.  RAV keeps the rows of the owned DoFs only
// (Sec. 4.3): owned = box nodes a in {2,3}^d (J = 2i + delta) and p_i.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cmath>
#include <type_traits>
#include <vector>

#include "box.cuh"
#include "common.cuh"
#include "fmt.cuh"

namespace rav {

// ---------------------------------------------------------------------------
// Factorisation: one block per subdomain.  Writes the requested fp64 rows in
// box coordinates, row-major: RAV rows = owned rows (NR), all rows otherwise (NC).
// MODE 0: owned rows; 1: all rows; 2: factored (owned rows of K^{-1}, w, 1/s).
template <int D, int MODE>
__global__ void __launch_bounds__(256) k_factor(Geo g, const int64_t* __restrict__ rp, const double* __restrict__ va,
                                                int64_t first, int64_t count, double* __restrict__ out,
                                                int* __restrict__ err) {
  using B = BoxT<D>;
  constexpr int NV = B::NV, NC = B::NC;
  constexpr bool ALL = MODE == 1;
  constexpr int NROW = ALL ? NC : B::NR;
  constexpr int NF = B::NF;
  constexpr int NRHS = 32;  // right-hand sides solved per batch
  extern __shared__ double sm[];
  double* K = sm;                  // NV x NV, lower triangle -> Cholesky factor
  double* bv = K + NV * NV;        // NV x D  (B column of p_i, node-major)
  double* w = bv + NV * D;         // NV x D  (A^{-1} b)
  double* Z = w + NV * D;          // NRHS x NV solutions
  __shared__ int valid[NV];
  __shared__ double s_inv;
  __shared__ int bad;
  const int64_t pl = blockIdx.x;
  if (pl >= count) return;
  const int64_t p = first + pl;
  int v[3] = {0, 0, 0};
  vertex_of(g, p, v);
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) bad = 0;
  for (int m = tid; m < NV; m += nt) {
    int a[3];
    box_tuple(D, m, a);
    valid[m] = box_node_valid(g, v, a);
  }
  __syncthreads();
  // K entries from velocity rows (component 0).  A free velocity row at node
  // J lists its velocity columns over the tensor range of the nodes of its cells.
  for (int e = tid; e < NV * NV; e += nt) {
    const int m = e / NV, n = e % NV;
    double val = (m == n) ? 1.0 : 0.0;
    if (valid[m] && valid[n]) {
      int am[3], an[3];
      box_tuple(D, m, am);
      box_tuple(D, n, an);
      int64_t Jm[3] = {0, 0, 0}, Jn[3] = {0, 0, 0};
      int64_t pos = 0, len = 1;
      bool in = true;
      for (int d = 0; d < D; ++d) {
        Jm[d] = 2 * v[d] - 2 + am[d];
        Jn[d] = 2 * v[d] - 2 + an[d];
      }
      for (int d = D - 1; d >= 0; --d) {
        int64_t lo, hi;
        if (Jm[d] & 1) { lo = Jm[d] - 1; hi = Jm[d] + 1; }
        else { lo = Jm[d] - 2 < 0 ? 0 : Jm[d] - 2; hi = Jm[d] + 2 > 2 * g.N ? 2 * g.N : Jm[d] + 2; }
        in &= (Jn[d] >= lo) & (Jn[d] <= hi);
        pos = pos * (hi - lo + 1) + (Jn[d] - lo);
        len *= hi - lo + 1;
      }
      val = 0.0;
      if (in) {
        const int64_t row = D * node_id(g, Jm);
        val = va[rp[row] + pos];
      }
    }
    K[m * NV + n] = val;
  }
  // b from the pressure row of p_i: columns = nodes [2v-2, 2v+2] (clipped) x components.
  {
    const int64_t prow = g.n_u + p;
    for (int e = tid; e < NV * D; e += nt) {
      const int m = e / D, c = e % D;
      double val = 0.0;
      if (valid[m]) {
        int a[3];
        box_tuple(D, m, a);
        int64_t pos = 0;
        for (int d = D - 1; d >= 0; --d) {
          const int64_t lo = 2 * v[d] - 2 < 0 ? 0 : 2 * v[d] - 2;
          const int64_t hi = 2 * v[d] + 2 > 2 * g.N ? 2 * g.N : 2 * v[d] + 2;
          pos = pos * (hi - lo + 1) + (2 * v[d] - 2 + a[d] - lo);
        }
        val = va[rp[prow] + pos * D + c];
      }
      bv[m * D + c] = val;
    }
  }
  __syncthreads();
  // Cholesky K = L L^T (lower triangle, right-looking).
  double dmax = 0.0;
  for (int m = 0; m < NV; ++m) dmax = fmax(dmax, fabs(K[m * NV + m]));
  for (int k = 0; k < NV; ++k) {
    if (tid == 0) {
      const double dkk = K[k * NV + k];
      if (!(dkk > 1e-14 * dmax)) { bad = 1; K[k * NV + k] = 1.0; }
      else K[k * NV + k] = sqrt(dkk);
    }
    __syncthreads();
    const double lkk = K[k * NV + k];
    for (int j = k + 1 + tid; j < NV; j += nt) K[j * NV + k] /= lkk;
    __syncthreads();
    const int rem = NV - k - 1;
    for (int e = tid; e < rem * rem; e += nt) {
      const int i = k + 1 + e / rem, j = k + 1 + e % rem;
      if (j <= i) K[i * NV + j] -= K[i * NV + k] * K[j * NV + k];
    }
    __syncthreads();
  }
  // Solves with the factor: warp r handles right-hand side r of the batch.
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  auto solve_rhs = [&](double* z) {
    for (int k = 0; k < NV; ++k) {  // L y = z
      const double yk = z[k] / K[k * NV + k];
      __syncwarp();
      if (lane == 0) z[k] = yk;
      for (int j = k + 1 + lane; j < NV; j += 32) z[j] -= K[j * NV + k] * yk;
      __syncwarp();
    }
    for (int k = NV - 1; k >= 0; --k) {  // L^T x = y
      const double xk = z[k] / K[k * NV + k];
      __syncwarp();
      if (lane == 0) z[k] = xk;
      for (int j = lane; j < k; j += 32) z[j] -= K[k * NV + j] * xk;
      __syncwarp();
    }
  };
  // w = K^{-1} b, one component per warp.
  for (int c = warp; c < D; c += nwarp) {
    double* z = Z + c * NV;
    for (int m = lane; m < NV; m += 32) z[m] = bv[m * D + c];
    __syncwarp();
    solve_rhs(z);
    for (int m = lane; m < NV; m += 32) w[m * D + c] = z[m];
  }
  __syncthreads();
  if (tid < 32) {
    double s = 0.0;
    for (int e = lane; e < NV * D; e += 32) s += bv[e] * w[e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const double sch = -s;
      double bmax = 0.0;
      for (int e = 0; e < NV * D; ++e) bmax = fmax(bmax, fabs(bv[e]));
      if (!(fabs(sch) > 1e-300) || bmax == 0.0) { bad = 1; s_inv = 0.0; }
      else s_inv = 1.0 / sch;
    }
  }
  __syncthreads();
  const double si = s_inv;
  if (MODE == 2) {
    // factored: rows of K^{-1} of the owned nodes, then w (node-major), then 1/s
    double* o = out + pl * (int64_t)NF;
    for (int q = warp; q < B::NON; q += nwarp) {
      const int m = (2 + (q & 1)) + 5 * (2 + ((q >> 1) & 1)) + (D == 3 ? 25 * (2 + ((q >> 2) & 1)) : 0);
      double* z = Z + q * NV;
      for (int n = lane; n < NV; n += 32) z[n] = (n == m) ? 1.0 : 0.0;
      __syncwarp();
      if (valid[m]) solve_rhs(z);
      __syncwarp();
      for (int n = lane; n < NV; n += 32) o[q * NV + n] = valid[m] && valid[n] ? z[n] : 0.0;
    }
    for (int e = tid; e < NV * D; e += nt) o[B::NON * NV + e] = w[e];
    if (tid == 0) o[NF - 1] = si;
    __syncthreads();
    if (tid == 0 && bad) atomicOr(err, 1);
    return;
  }
  double* orow = out + pl * (int64_t)NROW * NC;
  // Pressure row (last row in both layouts): (n,c') -> -w[n,c'] / s, (p,p) -> 1/s.
  for (int k = tid; k < NC; k += nt) orow[(int64_t)(NROW - 1) * NC + k] = k < NC - 1 ? -w[k] * si : si;
  // Velocity rows: row (m,c) = [delta_cc' Kinv[m,n] + w[m,c] w[n,c'] / s ; -w[m,c] / s].
  const int nnodes = ALL ? NV : B::NON;
  for (int r0 = 0; r0 < nnodes; r0 += NRHS) {
    const int nb = nnodes - r0 < NRHS ? nnodes - r0 : NRHS;
    __syncthreads();
    for (int r = warp; r < nb; r += nwarp) {
      const int q = r0 + r;  // row node index (ALL: box node; RAV: owned node)
      int m;
      if (ALL) m = q;
      else m = (2 + (q & 1)) + 5 * (2 + ((q >> 1) & 1)) + (D == 3 ? 25 * (2 + ((q >> 2) & 1)) : 0);
      double* z = Z + r * NV;
      for (int n = lane; n < NV; n += 32) z[n] = (n == m) ? 1.0 : 0.0;
      __syncwarp();
      if (valid[m]) solve_rhs(z);
      __syncwarp();
      for (int c = 0; c < D; ++c) {
        const int orw = ALL ? m * D + c : q * D + c;
        double* o = orow + (int64_t)orw * NC;
        const bool vm = valid[m];
        const double wm = w[m * D + c];
        for (int k = lane; k < NC; k += 32) {
          double val = 0.0;
          if (vm) {
            if (k < NC - 1) {
              const int n = k / D, c2 = k % D;
              val = (c2 == c ? z[n] : 0.0) + wm * w[k] * si;
              if (!valid[n]) val = 0.0;
            } else {
              val = -wm * si;
            }
          }
          o[k] = val;
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0 && bad) atomicOr(err, 1);
}

// Pack fp64 staging rows (box coordinates, row-major) into the RAV apply layout:
// unit u = subdomain * NCH + chunk (RB consecutive owned rows); units grouped
// by 32; element (u, jl, k) at ((u/32 * NC + k) * RB + jl) * 32 + u%32, so a
// warp reads 32 consecutive elements per (k, jl).  fp8 rows carry an fp32 scale
// max|row| / 448 (scale index (u/32 * RB + jl) * 32 + u%32).
template <int D, typename T>
__global__ void k_pack_rav(const double* __restrict__ stage, int64_t first, int64_t count, T* __restrict__ inv,
                           float* __restrict__ scale) {
  using B = BoxT<D>;
  constexpr int NC = B::NC, NR = B::NR, RB = B::RB, NCH = B::NCH;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (local unit, jl)
  if (t >= count * NR) return;
  const int64_t ul = t / RB;
  const int jl = (int)(t % RB);
  const int64_t pl = ul / NCH;
  const int h = (int)(ul % NCH);
  const int j = h * RB + jl;
  const int64_t u = first * NCH + ul;
  const int64_t G = u >> 5;
  const int lane = (int)(u & 31);
  const double* row = stage + (pl * NR + j) * (int64_t)NC;
  double s = 1.0;
  if (Fmt<T>::scaled) {
    double m = 0.0;
    for (int k = 0; k < NC; ++k) m = fmax(m, fabs(row[k]));
    s = m == 0.0 ? 1.0 : (double)(float)(m / 448.0);
    scale[(G * RB + jl) * 32 + lane] = (float)s;
  }
  for (int k = 0; k < NC; ++k) inv[((G * NC + k) * RB + jl) * 32 + lane] = Fmt<T>::enc(row[k] / s);
}

// Full inverses (AV, MV): per subdomain column-major NC x NC (element (j,k) at k*NC + j).
template <int D>
__global__ void k_pack_full(const double* __restrict__ stage, int64_t first, int64_t count, double* __restrict__ inv) {
  constexpr int NC = BoxT<D>::NC;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count * NC * NC) return;
  const int64_t pl = t / (NC * NC);
  const int e = (int)(t % (NC * NC));
  const int j = e / NC, k = e % NC;
  inv[(first + pl) * (int64_t)NC * NC + (int64_t)k * NC + j] = stage[t];
}

// ---------------------------------------------------------------------------
// RAV apply (Eq. 13): one thread per unit; gathers the NC residual entries of
// its subdomain, forms RB owned rows of L_i^{-1} r_i and adds omega_i times
// them to the owned DoFs of x.  Owned DoFs of different subdomains are
// disjoint, so the writes need no atomics.
// The residual arrives in the accumulation type: fp64 for fp64 storage, else
// already rounded to fp32 (once per entry, not once per read).

template <int D, typename T>
__global__ void __launch_bounds__(128) k_rav_apply(Geo g, const T* __restrict__ inv, const float* __restrict__ scale,
                                                   const double* __restrict__ omega, const AccT<T>* __restrict__ r,
                                                   double* __restrict__ x, int64_t units) {
  using B = BoxT<D>;
  constexpr int NC = B::NC, RB = B::RB, NCH = B::NCH;
  using Acc = AccT<T>;
  __shared__ float lut[256];
  if (Fmt<T>::scaled) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
      __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)i, __NV_E4M3);
      lut[i] = __half2float(__half(h));
    }
    __syncthreads();
  }
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= units) return;
  const int64_t p = u / NCH;
  const int h = (int)(u % NCH);
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  const int M = (int)g.M;
  int alo[3] = {0, 0, 0}, ahi[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d) {
    if (d < D) {
      alo[d] = 2 - 2 * v[d] > 0 ? 2 - 2 * v[d] : 0;
      ahi[d] = 2 * g.N - 2 * v[d] + 2 < 4 ? 2 * g.N - 2 * v[d] + 2 : 4;
    }
  }
  int64_t base = 0;
  for (int d = D - 1; d >= 0; --d) base = base * M + (2 * v[d] - 2);
  base *= D;
  const T* ip = inv + ((u >> 5) * NC * RB) * 32 + (u & 31);
  Acc acc[RB];
#pragma unroll
  for (int j = 0; j < RB; ++j) acc[j] = 0;
  int k = 0;
  for (int a2 = 0; a2 < (D == 3 ? 5 : 1); ++a2) {
    const bool v2 = D == 2 || (a2 >= alo[2] && a2 <= ahi[2]);
    for (int a1 = 0; a1 < 5; ++a1) {
      const bool v1 = v2 && a1 >= alo[1] && a1 <= ahi[1];
      const int64_t rowoff = base + (int64_t)D * M * (a1 + (int64_t)M * a2);
#pragma unroll
      for (int a0 = 0; a0 < 5; ++a0) {
        const bool vv = v1 && a0 >= alo[0] && a0 <= ahi[0];
        Acc rn[D];
        if constexpr (D == 2 && std::is_same<Acc, float>::value) {
          // the two fp32 components of a node are one aligned 8-byte load
          float2 rv = make_float2(0.f, 0.f);
          if (vv) rv = *reinterpret_cast<const float2*>(r + rowoff + 2 * a0);
          rn[0] = rv.x;
          rn[1] = rv.y;
        } else {
#pragma unroll
          for (int c = 0; c < D; ++c) rn[c] = vv ? r[rowoff + D * a0 + c] : (Acc)0;
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const Acc ra = rn[c];
#pragma unroll
          for (int j = 0; j < RB; ++j) acc[j] += (Acc)Fmt<T>::dec(ip[(k * RB + j) * 32], lut) * ra;
          ++k;
        }
      }
    }
  }
  {
    const Acc ra = r[g.n_u + p];
#pragma unroll
    for (int j = 0; j < RB; ++j) acc[j] += (Acc)Fmt<T>::dec(ip[(k * RB + j) * 32], lut) * ra;
  }
  const double om = omega[p];
#pragma unroll
  for (int jl = 0; jl < RB; ++jl) {
    const int j = h * RB + jl;
    Acc y = acc[jl];
    if (Fmt<T>::scaled) y *= scale[((u >> 5) * RB + jl) * 32 + (u & 31)];
    if (j < B::NR - 1) {
      const int q = j / D, c = j % D;
      int64_t J[3] = {0, 0, 0};
      bool ok = true;
      for (int d = 0; d < D; ++d) {
        J[d] = 2 * v[d] + ((q >> d) & 1);
        ok &= (J[d] >= 1) & (J[d] <= 2 * g.N - 1);
      }
      if (ok) x[D * node_id_t<D>(g, J) + c] += om * (double)y;
    } else {
      x[g.n_u + p] += om * (double)y;
    }
  }
}

// ---------------------------------------------------------------------------
// Factored RAV storage.  Rows of K^{-1} of the owned nodes: unit u = subdomain
// * 2^d + owned node q, element (u, n) at ((u/32) * NV + n) * 32 + u%32.
// w (node-major, NV*D) and 1/s: per subdomain, contiguous (NV*D + 1 values).
// Stored as T (fp64, or rounded to nearest even into fp32 / bf16).
// K^{-1} rows grouped by G = 2^lg units: element (u, n) at
// ((u / G) NV + n) G + u % G, so the G units of a warp read G consecutive values.
template <int D, typename T>
__global__ void k_pack_fact(const double* __restrict__ stage, int64_t first, int64_t count,
                            T* __restrict__ kinv, T* __restrict__ ws, int lg) {
  using B = BoxT<D>;
  constexpr int NV = B::NV, NON = B::NON, NF = B::NF, NWS = D * NV + 1;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < count * NON) {
    const int64_t pl = t / NON;
    const int q = (int)(t % NON);
    const int64_t u = (first + pl) * NON + q;
    const double* src = stage + pl * NF + q * NV;
    const int64_t G = int64_t(1) << lg;
    T* dst = kinv + ((u >> lg) * NV) * G + (u & (G - 1));
    for (int n = 0; n < NV; ++n) dst[n * G] = Fmt<T>::enc(src[n]);
  }
  if (t < count * NWS) {
    const int64_t pl = t / NWS;
    const int e = (int)(t % NWS);
    ws[(first + pl) * NWS + e] = Fmt<T>::enc(stage[pl * NF + NON * NV + e]);
  }
}

// Moves K^{-1} rows from grouping 2^ls to grouping 2^ld (one thread per element).
template <typename T>
__global__ void k_regroup(const T* __restrict__ src, T* __restrict__ dst, int64_t units, int nv, int ls, int ld) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= units * nv) return;
  const int64_t u = e / nv;
  const int n = (int)(e % nv);
  const int64_t Gs = int64_t(1) << ls, Gd = int64_t(1) << ld;
  dst[((u >> ld) * nv + n) * Gd + (u & (Gd - 1))] = src[((u >> ls) * nv + n) * Gs + (u & (Gs - 1))];
}

// RAV apply with the factored inverse (Eq. 13 via the block form of L_i^{-1}):
//   tau = (1/s) (w^T r_u - r_p),
//   y(m,c) = sum_n K^{-1}[m,n] r(n,c) + w(m,c) tau   for the owned nodes m,
//   y_p = -tau;   x[owned] += omega_i y.
// One unit per owned node (2^d per subdomain), S threads per unit: a warp
// holds G = 32/S units, lane = s G + j for split s and unit j; split s sums the
// box nodes n = s, s+S, ... and the S partial sums meet by shuffles (offsets
// G, 2G, ...).  w^T r_u is split over all 2^d S threads of the subdomain.
// More splits keep small levels busy; the storage grouping follows G.
// Reduced storage types accumulate in fp32 and read the fp32-rounded residual;
// fp64 storage accumulates in fp64.
// Register caps (blocks of 128 per SM): 3-D reduced storage at 32 registers,
// so that a 32^3 level's units fit in one wave; the others at what they need
// without spilling (about 40 in 2-D, 48 in 3-D fp64).
template <int D, typename T>
constexpr int fact_min_blocks() {
  return D == 3 ? (std::is_same<T, double>::value ? 10 : 16) : 12;
}

template <int D, typename T, int S>
__global__ void __launch_bounds__(128, fact_min_blocks<D, T>()) k_rav_apply_fact(Geo g, const T* __restrict__ kinv,
                                                        const T* __restrict__ ws,
                                                        const double* __restrict__ omega,
                                                        const AccT<T>* __restrict__ r, double* __restrict__ x,
                                                        int64_t units) {
  using B = BoxT<D>;
  constexpr int NV = B::NV, NON = B::NON, NWS = D * NV + 1, G = 32 / S;
  static_assert(G % NON == 0, "a warp holds whole subdomains");
  using A = AccT<T>;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = (int)(t0 & 31);
  const int sp = lane / G;
  const int64_t u = (t0 >> 5) * G + (lane % G);
  // warps past the last unit own no storage; the others stay whole (their
  // shuffles need every lane), idle lanes computing on subdomain 0
  if ((t0 >> 5) * G >= units) return;
  const bool active = u < units;
  const int64_t p = active ? u / NON : 0;
  const int q = (int)(u & (NON - 1));
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  const int M = (int)g.M;
  int alo[3] = {0, 0, 0}, ahi[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    alo[d] = 2 - 2 * v[d] > 0 ? 2 - 2 * v[d] : 0;
    ahi[d] = 2 * g.N - 2 * v[d] + 2 < 4 ? 2 * g.N - 2 * v[d] + 2 : 4;
  }
  int64_t base = 0;
#pragma unroll
  for (int d = D - 1; d >= 0; --d) base = base * M + (2 * v[d] - 2);
  base *= D;
  const T* kp = kinv + ((u / G) * NV) * G + (u % G);
  A y[D];
#pragma unroll
  for (int c = 0; c < D; ++c) y[c] = 0;
  if (S == 1) {
    int n = 0;
    for (int a2 = 0; a2 < (D == 3 ? 5 : 1); ++a2) {
      const bool v2 = D == 2 || (a2 >= alo[2] && a2 <= ahi[2]);
      for (int a1 = 0; a1 < 5; ++a1) {
        const bool v1 = v2 && a1 >= alo[1] && a1 <= ahi[1];
        const int64_t rowoff = base + (int64_t)D * M * (a1 + (int64_t)M * a2);
#pragma unroll
        for (int a0 = 0; a0 < 5; ++a0) {
          const bool vv = v1 && a0 >= alo[0] && a0 <= ahi[0];
          const A kq = (A)Fmt<T>::dec(ld_stream(kp + n * G), nullptr);
          if constexpr (D == 2 && std::is_same<A, float>::value) {
            // the two fp32 components of a node are one aligned 8-byte load
            float2 rv = make_float2(0.f, 0.f);
            if (vv) rv = *reinterpret_cast<const float2*>(r + rowoff + 2 * a0);
            y[0] += kq * rv.x;
            y[1] += kq * rv.y;
          } else {
#pragma unroll
            for (int c = 0; c < D; ++c) y[c] += kq * (vv ? r[rowoff + D * a0 + c] : (A)0);
          }
          ++n;
        }
      }
    }
  } else {
    for (int n = sp; n < NV; n += S) {
      const int a0 = n % 5, a1 = (n / 5) % 5, a2 = D == 3 ? n / 25 : 0;
      bool vv = a0 >= alo[0] && a0 <= ahi[0] && a1 >= alo[1] && a1 <= ahi[1];
      if (D == 3) vv = vv && a2 >= alo[2] && a2 <= ahi[2];
      const int64_t off = base + (int64_t)D * (a0 + (int64_t)M * (a1 + (int64_t)M * a2));
      const A kq = (A)Fmt<T>::dec(ld_stream(kp + n * G), nullptr);
#pragma unroll
      for (int c = 0; c < D; ++c) y[c] += kq * (vv ? r[off + c] : (A)0);
    }
#pragma unroll
    for (int o = G; o < 32; o <<= 1)
#pragma unroll
      for (int c = 0; c < D; ++c) y[c] += __shfl_xor_sync(0xffffffffu, y[c], o);
  }
  // partial w^T r_u over the box nodes n = q + 2^d s, q + 2^d s + 2^d S, ...
  const T* wp = ws + p * NWS;
  A t = 0;
  for (int m = q + NON * sp; m < NV; m += NON * S) {
    const int a0 = m % 5, a1 = (m / 5) % 5, a2 = D == 3 ? m / 25 : 0;
    bool vv = a0 >= alo[0] && a0 <= ahi[0] && a1 >= alo[1] && a1 <= ahi[1];
    if (D == 3) vv = vv && a2 >= alo[2] && a2 <= ahi[2];
    if (vv) {
      const int64_t off = base + (int64_t)D * (a0 + (int64_t)M * (a1 + (int64_t)M * a2));
#pragma unroll
      for (int c = 0; c < D; ++c) t += (A)Fmt<T>::dec(wp[m * D + c], nullptr) * r[off + c];
    }
  }
#pragma unroll
  for (int o = NON / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
#pragma unroll
  for (int o = G; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (!active || sp != 0) return;
  const A tau = (A)Fmt<T>::dec(wp[NWS - 1], nullptr) * (t - r[g.n_u + p]);
  const double om = omega[p];
  int64_t J[3] = {0, 0, 0};
  bool ok = true;
  int mq = 0;
#pragma unroll
  for (int d = D - 1; d >= 0; --d) {
    const int dl = (q >> d) & 1;
    J[d] = 2 * v[d] + dl;
    ok &= (J[d] >= 1) & (J[d] <= 2 * g.N - 1);
    mq = mq * 5 + 2 + dl;
  }
  if (ok) {
    const int64_t dof = D * node_id_t<D>(g, J);
#pragma unroll
    for (int c = 0; c < D; ++c) x[dof + c] += om * (double)(y[c] + (A)Fmt<T>::dec(wp[mq * D + c], nullptr) * tau);
  }
  if (q == 0) x[g.n_u + p] += om * (double)-tau;
}

// ---------------------------------------------------------------------------
// Full-inverse subdomain solve shared by AV and MV: one warp per subdomain,
// rloc in shared memory, y = L_i^{-1} rloc with the column-major inverse.
template <int D>
__device__ void warp_full_solve(const double* __restrict__ Inv, const double* rloc, double* y) {
  constexpr int NC = BoxT<D>::NC;
  const int lane = threadIdx.x & 31;
  for (int j = lane; j < NC; j += 32) {
    double s = 0.0;
    for (int k = 0; k < NC; ++k) s += Inv[(int64_t)k * NC + j] * rloc[k];
    y[j] = s;
  }
  __syncwarp();
}

// Global DoF of box position k of the subdomain at vertex v (-1 if not in it).
template <int D>
__device__ __forceinline__ int64_t box_dof(const Geo& g, const int* v, int64_t p, int k) {
  constexpr int NC = BoxT<D>::NC;
  if (k == NC - 1) return g.n_u + p;
  int a[3];
  box_tuple(D, k / D, a);
  if (!box_node_valid(g, v, a)) return -1;
  int64_t J[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) J[d] = 2 * v[d] - 2 + a[d];
  return D * node_id(g, J) + k % D;
}

// AV (Eq. 12), step 1: corr[p][k] = omega_p (L_p^{-1} r_p)_k for every box position.
template <int D>
__global__ void k_av_corr(Geo g, const double* __restrict__ inv, const double* __restrict__ omega,
                          const double* __restrict__ r, double* __restrict__ corr) {
  constexpr int NC = BoxT<D>::NC;
  constexpr int WPB = 4;
  __shared__ double rl[WPB][NC], yl[WPB][NC];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = blockIdx.x * (int64_t)WPB + wi;
  if (p >= g.n_p) return;
  int v[3] = {0, 0, 0};
  vertex_of(g, p, v);
  for (int k = lane; k < NC; k += 32) {
    const int64_t dof = box_dof<D>(g, v, p, k);
    rl[wi][k] = dof >= 0 ? r[dof] : 0.0;
  }
  __syncwarp();
  warp_full_solve<D>(inv + p * (int64_t)NC * NC, rl[wi], yl[wi]);
  const double om = omega[p];
  for (int k = lane; k < NC; k += 32) corr[p * NC + k] = om * yl[wi][k];
}

// AV, step 2: x[dof] += sum over the subdomains containing dof (ascending) of corr.
template <int D>
__global__ void k_av_gather(Geo g, const double* __restrict__ corr, double* __restrict__ x) {
  constexpr int NC = BoxT<D>::NC;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  if (i >= g.n_u) {
    x[i] += corr[(i - g.n_u) * NC + NC - 1];
    return;
  }
  int64_t I[3] = {0, 0, 0};
  int c;
  vel_node(g, i, I, c);
  if (node_on_boundary(g, I)) return;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) {
    lo[d] = (int)((I[d] - 1) >> 1);  // vertices v with 2v-2 <= I <= 2v+2
    hi[d] = (int)((I[d] + 2) >> 1);
    lo[d] = lo[d] < 0 ? 0 : lo[d];
    hi[d] = hi[d] > g.N ? g.N : hi[d];
  }
  double s = 0.0;
  for (int v2 = (D == 3 ? lo[2] : 0); v2 <= (D == 3 ? hi[2] : 0); ++v2)
    for (int v1 = lo[1]; v1 <= hi[1]; ++v1)
      for (int v0 = lo[0]; v0 <= hi[0]; ++v0) {
        const int vv[3] = {v0, v1, v2};
        int64_t p = 0;
        int m = 0;
        for (int d = D - 1; d >= 0; --d) {
          p = p * (g.N + 1) + vv[d];
          m = m * 5 + (int)(I[d] - (2 * vv[d] - 2));
        }
        s += corr[p * NC + m * D + c];
      }
  x[i] += s;
}

// MV (Eq. 11 with the residual refresh of Eq. 15) over one colour class:
// subdomains whose vertices agree mod 4 on every axis touch disjoint DoFs and
// read no DoF another one of the class writes, so the class is processed in
// parallel and equals the sequential sweep over it.
template <int D>
__global__ void k_mv_colour(Geo g, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ va, const double* __restrict__ inv,
                            const double* __restrict__ omega, const double* __restrict__ b, double* __restrict__ x,
                            int colour) {
  constexpr int NC = BoxT<D>::NC;
  constexpr int WPB = 4;
  __shared__ double rl[WPB][NC], yl[WPB][NC];
  __shared__ int64_t dl[WPB][NC];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // enumerate the vertices of this colour: v_a = col_a + 4 t_a
  int col[3] = {colour & 3, (colour >> 2) & 3, (colour >> 4) & 3};
  int cnt[3] = {1, 1, 1};
  int64_t tot = 1;
  for (int d = 0; d < D; ++d) {
    cnt[d] = col[d] <= g.N ? (g.N - col[d]) / 4 + 1 : 0;
    tot *= cnt[d];
  }
  const int64_t t = blockIdx.x * (int64_t)WPB + wi;
  if (t >= tot) return;
  int v[3] = {0, 0, 0};
  {
    int64_t tt = t;
    for (int d = 0; d < D; ++d) { v[d] = col[d] + 4 * (int)(tt % cnt[d]); tt /= cnt[d]; }
  }
  int64_t p = 0;
  for (int d = D - 1; d >= 0; --d) p = p * (g.N + 1) + v[d];
  for (int k = lane; k < NC; k += 32) {
    const int64_t dof = box_dof<D>(g, v, p, k);
    dl[wi][k] = dof;
    double s = 0.0;
    if (dof >= 0) {
      s = b[dof];
      for (int64_t q = rp[dof]; q < rp[dof + 1]; ++q) s -= va[q] * x[ci[q]];
    }
    rl[wi][k] = s;
  }
  __syncwarp();
  warp_full_solve<D>(inv + p * (int64_t)NC * NC, rl[wi], yl[wi]);
  const double om = omega[p];
  for (int k = lane; k < NC; k += 32)
    if (dl[wi][k] >= 0) x[dl[wi][k]] += om * yl[wi][k];
}

// ---------------------------------------------------------------------------
// Inspection: compact (sorted) subdomain lists and the stored rows expanded.
template <int D>
__global__ void k_patch_count(Geo g, int32_t* __restrict__ cnt) {
  constexpr int NC = BoxT<D>::NC;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= g.n_p) return;
  int v[3] = {0, 0, 0};
  vertex_of(g, p, v);
  int c = 0;
  for (int k = 0; k < NC; k += D) {
    if (k == NC - 1) { ++c; break; }
    int a[3];
    box_tuple(D, k / D, a);
    if (box_node_valid(g, v, a)) c += D;
  }
  cnt[p] = c;
}
template <int D>
__global__ void k_patch_list(Geo g, const int32_t* __restrict__ off, int32_t* __restrict__ dofs) {
  constexpr int NC = BoxT<D>::NC;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= g.n_p) return;
  int v[3] = {0, 0, 0};
  vertex_of(g, p, v);
  int32_t pos = off[p];
  for (int k = 0; k < NC; ++k) {
    const int64_t dof = box_dof<D>(g, v, p, k);
    if (dof >= 0) dofs[pos++] = (int32_t)dof;
  }
}
// owner(velocity DoF at node I) = vertex floor(I/2) (Q2-Q1) or vertex I
// (Q1-Q1); owner(p_i) = i; Dirichlet -1.
__global__ void k_owner(Geo g, int32_t* __restrict__ owner) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  if (i >= g.n_u) { owner[i] = (int32_t)(i - g.n_u); return; }
  int64_t I[3] = {0, 0, 0};
  int c;
  vel_node(g, i, I, c);
  if (node_on_boundary(g, I)) { owner[i] = -1; return; }
  int64_t v[3];
  for (int d = 0; d < g.dim; ++d) v[d] = g.q == 1 ? I[d] : I[d] >> 1;
  owner[i] = (int32_t)vert_id(g, v);
}
__global__ void k_scan_i32(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ off) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int32_t a = 0;
    for (int64_t i = 0; i < n; ++i) { off[i] = a; a += cnt[i]; }
    off[n] = a;
  }
}

// Expanded stored rows for subdomains [first, first+count): out[p][j][k] in
// compact sorted order, padded to rows_max x cols_max.
template <int D, typename T>
__global__ void k_export_rav(Geo g, const T* __restrict__ inv, const float* __restrict__ scale, int64_t first,
                             int64_t count, double* __restrict__ out) {
  using B = BoxT<D>;
  constexpr int NC = B::NC, NR = B::NR, RB = B::RB, NCH = B::NCH;
  __shared__ float lut[256];
  __shared__ int colmap[NC], rowmap[NR];
  __shared__ int ncol, nrow;
  if (Fmt<T>::scaled) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
      __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)i, __NV_E4M3);
      lut[i] = __half2float(__half(h));
    }
  }
  const int64_t p = first + blockIdx.x;
  int v[3] = {0, 0, 0};
  vertex_of(g, p, v);
  if (threadIdx.x == 0) {
    int c = 0;
    for (int k = 0; k < NC; ++k)
      if (box_dof<D>(g, v, p, k) >= 0) colmap[c++] = k;
    ncol = c;
    int rr = 0;
    for (int j = 0; j < NR; ++j) {
      int k;
      if (j == NR - 1) k = NC - 1;
      else {
        const int q = j / D;
        const int m = (2 + (q & 1)) + 5 * (2 + ((q >> 1) & 1)) + (D == 3 ? 25 * (2 + ((q >> 2) & 1)) : 0);
        k = m * D + j % D;
      }
      if (box_dof<D>(g, v, p, k) >= 0) rowmap[rr++] = j;
    }
    nrow = rr;
  }
  __syncthreads();
  double* o = out + blockIdx.x * (int64_t)NR * NC;
  for (int e = threadIdx.x; e < NR * NC; e += blockDim.x) {
    const int jr = e / NC, kc = e % NC;
    double val = 0.0;
    if (jr < nrow && kc < ncol) {
      const int j = rowmap[jr], k = colmap[kc];
      const int64_t u = p * NCH + j / RB;
      const int jl = j % RB;
      val = (double)Fmt<T>::dec(inv[(((u >> 5) * NC + k) * RB + jl) * 32 + (u & 31)], lut);
      if (Fmt<T>::scaled) val *= (double)scale[((u >> 5) * RB + jl) * 32 + (u & 31)];
    }
    o[e] = val;
  }
}
// Owned rows of L_i^{-1} rebuilt from the factored storage:
// (m,c | n,c') = delta_cc' K^{-1}[m,n] + w(m,c) w(n,c') / s,  (m,c | p) = -w(m,c) / s,
// (p | n,c') = -w(n,c') / s,  (p | p) = 1 / s.
template <int D, typename T>
__global__ void k_export_fact(Geo g, const T* __restrict__ kinv, const T* __restrict__ ws, int64_t first,
                              int64_t count, double* __restrict__ out, int lg) {
  using B = BoxT<D>;
  constexpr int NC = B::NC, NR = B::NR, NV = B::NV, NON = B::NON, NWS = D * NV + 1;
  __shared__ int colmap[NC], rowmap[NR];
  __shared__ int ncol, nrow;
  const int64_t p = first + blockIdx.x;
  int v[3] = {0, 0, 0};
  vertex_of(g, p, v);
  if (threadIdx.x == 0) {
    int c = 0;
    for (int k = 0; k < NC; ++k)
      if (box_dof<D>(g, v, p, k) >= 0) colmap[c++] = k;
    ncol = c;
    int rr = 0;
    for (int j = 0; j < NR; ++j) {
      int k;
      if (j == NR - 1) k = NC - 1;
      else {
        const int q = j / D;
        const int m = (2 + (q & 1)) + 5 * (2 + ((q >> 1) & 1)) + (D == 3 ? 25 * (2 + ((q >> 2) & 1)) : 0);
        k = m * D + j % D;
      }
      if (box_dof<D>(g, v, p, k) >= 0) rowmap[rr++] = j;
    }
    nrow = rr;
  }
  __syncthreads();
  const T* wp = ws + p * NWS;
  const double sig = (double)Fmt<T>::dec(wp[NWS - 1], nullptr);
  double* o = out + blockIdx.x * (int64_t)NR * NC;
  for (int e = threadIdx.x; e < NR * NC; e += blockDim.x) {
    const int jr = e / NC, kc = e % NC;
    double val = 0.0;
    if (jr < nrow && kc < ncol) {
      const int j = rowmap[jr], k = colmap[kc];
      const bool prow = j == NR - 1, pcol = k == NC - 1;
      if (prow && pcol) {
        val = sig;
      } else if (prow) {
        val = -(double)Fmt<T>::dec(wp[k], nullptr) * sig;
      } else {
        const int q = j / D, c = j % D;
        const int m = (2 + (q & 1)) + 5 * (2 + ((q >> 1) & 1)) + (D == 3 ? 25 * (2 + ((q >> 2) & 1)) : 0);
        const double wm = (double)Fmt<T>::dec(wp[m * D + c], nullptr);
        if (pcol) {
          val = -wm * sig;
        } else {
          const int n = k / D, c2 = k % D;
          const int64_t u = p * NON + q;
          const int64_t G = int64_t(1) << lg;
          const double kq = (double)Fmt<T>::dec(kinv[((u >> lg) * NV + n) * G + (u & (G - 1))], nullptr);
          val = (c2 == c ? kq : 0.0) + wm * (double)Fmt<T>::dec(wp[k], nullptr) * sig;
        }
      }
    }
    o[e] = val;
  }
}

template <int D>
__global__ void k_export_full(Geo g, const double* __restrict__ inv, int64_t first, int64_t count,
                              double* __restrict__ out) {
  constexpr int NC = BoxT<D>::NC;
  __shared__ int colmap[NC];
  __shared__ int ncol;
  const int64_t p = first + blockIdx.x;
  int v[3] = {0, 0, 0};
  vertex_of(g, p, v);
  if (threadIdx.x == 0) {
    int c = 0;
    for (int k = 0; k < NC; ++k)
      if (box_dof<D>(g, v, p, k) >= 0) colmap[c++] = k;
    ncol = c;
  }
  __syncthreads();
  double* o = out + blockIdx.x * (int64_t)NC * NC;
  for (int e = threadIdx.x; e < NC * NC; e += blockDim.x) {
    const int jr = e / NC, kc = e % NC;
    double val = 0.0;
    if (jr < ncol && kc < ncol) val = inv[p * (int64_t)NC * NC + (int64_t)colmap[kc] * NC + colmap[jr]];
    o[e] = val;
  }
}

// ---------------------------------------------------------------------------
// Stabilised Q1-Q1 subdomains (Sec. 3 on the paper's own element): subdomain
// i = p_i plus the free velocity DoFs of the 3^d vertices J = v - 1 + a,
// a in [0,3)^d (box node m = a0 + 3 a1 + 9 a2, ascending m = ascending DoF);
// it owns the velocity DoFs of vertex v itself (m = CEN) and p_i.  The local
// system is [K (x) I_d, b; b^T, c] with K the scalar velocity block, b the
// pressure row's velocity entries and c its diagonal (the stabilisation of
// Eq. 8), so with w_c = K^{-1} b_c and s = c - sum_c b_c^T w_c the owned rows
// of L_i^{-1} follow from the centre row of K^{-1}, w and 1/s.  Stored per
// subdomain, structure of arrays (value k of subdomain p at k np + p):
//   k in [0, NV): row CEN of K^{-1};  [NV, NV + d NV): w (node-major);  last: 1/s.
template <int D>
struct Q1Box {
  static constexpr int NV = D == 2 ? 9 : 27;  // box vertices
  static constexpr int NC = D * NV + 1;       // box positions
  static constexpr int NR = D + 1;            // owned rows
  static constexpr int NF = NV * (D + 1) + 1; // stored values per subdomain
  static constexpr int CEN = D == 2 ? 4 : 13; // the subdomain's own vertex
};
__device__ __forceinline__ void q1_tuple(int m, int* a) {
  a[0] = m % 3;
  a[1] = (m / 3) % 3;
  a[2] = m / 9;
}
// Box vertex m of subdomain v is a free velocity node: 1 <= v - 1 + a <= N - 1 on every axis.
template <int D>
__device__ __forceinline__ bool q1_free(const Geo& g, const int* v, int m) {
  int a[3];
  q1_tuple(m, a);
  bool ok = true;
#pragma unroll
  for (int d = 0; d < D; ++d) ok &= (v[d] - 1 + a[d] >= 1) & (v[d] - 1 + a[d] <= g.N - 1);
  return ok;
}

// One warp per subdomain: gather K, b and c from the CSR rows, Cholesky
// K = L L^T, then one lane per right-hand side.  RAV (FULL = false, 4 warps
// per block): solve for K^{-1} e_CEN and K^{-1} b_c and write the NF stored
// values in fp64 to out (SoA, stride np).  AV/MV (FULL = true): solve for
// every column of K^{-1} and the w_c, and write the whole L_i^{-1} over the
// box positions (velocity m d + c, pressure last; identity at absent
// positions), column-major, NC x NC per subdomain.
template <int D, bool FULL>
__global__ void __launch_bounds__(128) k_factor_q1(Geo g, const int64_t* __restrict__ rp,
                                                   const double* __restrict__ va, int64_t np,
                                                   double* __restrict__ out, int* __restrict__ err) {
  using B = Q1Box<D>;
  constexpr int NV = B::NV, NF = B::NF, NC = B::NC;
  constexpr int NE = FULL ? NV : 1;  // unit right-hand sides
  constexpr int NRHS = NE + D;
  constexpr int WPB = (FULL && D == 3) ? 2 : 4;
  static_assert(NRHS <= 32, "one lane per right-hand side");
  __shared__ double sK[WPB][NV * NV];
  __shared__ double sB[WPB][NV * D];
  __shared__ double sZ[WPB][NRHS * NV];
  __shared__ int sv[WPB][NV];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w >= WPB) return;
  const int64_t p = blockIdx.x * (int64_t)WPB + w;
  if (p >= np) return;  // whole warps
  double* K = sK[w];
  double* b = sB[w];
  double* Z = sZ[w];
  int* valid = sv[w];
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  const int64_t N1 = g.N + 1;
  for (int m = lane; m < NV; m += 32) valid[m] = q1_free<D>(g, v, m);
  __syncwarp();
  // K from the component-0 rows of the free box vertices: a free row J lists
  // its velocity columns over [J-1, J+1] per axis (all inside the grid)
  for (int e = lane; e < NV * NV; e += 32) {
    const int m = e / NV, n = e % NV;
    double val = m == n ? 1.0 : 0.0;
    if (valid[m] && valid[n]) {
      int am[3], an[3];
      q1_tuple(m, am);
      q1_tuple(n, an);
      bool in = true;
      int pos = 0;
      int64_t jm = 0;
      for (int d = D - 1; d >= 0; --d) {
        const int dj = an[d] - am[d];
        in &= dj >= -1 && dj <= 1;
        pos = pos * 3 + (dj + 1);
        jm = jm * N1 + (v[d] - 1 + am[d]);
      }
      val = in ? va[rp[D * jm] + pos] : 0.0;
    }
    K[e] = val;
  }
  // b from the pressure row of p: velocity columns over [v-1, v+1] clipped, D per vertex
  const int64_t prow = g.n_u + p;
  int lo[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
  for (int d = 0; d < D; ++d) {
    lo[d] = v[d] - 1 < 0 ? 0 : v[d] - 1;
    const int hi = v[d] + 1 > g.N ? g.N : v[d] + 1;
    ext[d] = hi - lo[d] + 1;
  }
  for (int e = lane; e < NV * D; e += 32) {
    const int m = e / D, c = e % D;
    double val = 0.0;
    if (valid[m]) {
      int a[3];
      q1_tuple(m, a);
      int pos = 0;
      for (int d = D - 1; d >= 0; --d) pos = pos * ext[d] + (v[d] - 1 + a[d] - lo[d]);
      val = va[rp[prow] + pos * D + c];
    }
    b[e] = val;
  }
  double cdiag = 0.0;
  if (lane == 0) {
    int cnt = 1, pos = 0;
    for (int d = D - 1; d >= 0; --d) {
      cnt *= ext[d];
      pos = pos * ext[d] + (v[d] - lo[d]);
    }
    cdiag = va[rp[prow] + D * cnt + pos];
  }
  __syncwarp();
  double dmax = 0.0;
  for (int m = lane; m < NV; m += 32) dmax = fmax(dmax, fabs(K[m * NV + m]));
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  int bad = 0;
  for (int k = 0; k < NV; ++k) {
    if (lane == 0) {
      const double dkk = K[k * NV + k];
      if (!(dkk > 1e-14 * dmax)) { bad = 1; K[k * NV + k] = 1.0; }
      else K[k * NV + k] = sqrt(dkk);
    }
    __syncwarp();
    const double lkk = K[k * NV + k];
    for (int j = k + 1 + lane; j < NV; j += 32) K[j * NV + k] /= lkk;
    __syncwarp();
    const int rem = NV - k - 1;
    for (int e = lane; e < rem * rem; e += 32) {
      const int i = k + 1 + e / rem, j = k + 1 + e % rem;
      if (j <= i) K[i * NV + j] -= K[i * NV + k] * K[j * NV + k];
    }
    __syncwarp();
  }
  if (lane < NRHS) {  // right-hand side lane: unit vectors (e_CEN, or all), then b_0 .. b_{D-1}
    double* z = Z + lane * NV;
    const int eidx = FULL ? lane : B::CEN;
    for (int i = 0; i < NV; ++i) {
      double acc = lane < NE ? (i == eidx ? 1.0 : 0.0) : b[i * D + lane - NE];
      for (int j = 0; j < i; ++j) acc -= K[i * NV + j] * z[j];
      z[i] = acc / K[i * NV + i];
    }
    for (int i = NV - 1; i >= 0; --i) {
      double acc = z[i];
      for (int j = i + 1; j < NV; ++j) acc -= K[j * NV + i] * z[j];
      z[i] = acc / K[i * NV + i];
    }
  }
  __syncwarp();
  double sinv = 0.0;
  if (lane == 0) {
    double sch = cdiag;
    for (int c = 0; c < D; ++c)
      for (int m = 0; m < NV; ++m) sch -= b[m * D + c] * Z[(NE + c) * NV + m];
    if (!(fabs(sch) > 0.0) || !isfinite(sch)) bad = 1;
    else sinv = 1.0 / sch;
  }
  sinv = __shfl_sync(0xffffffffu, sinv, 0);
  bad = __shfl_sync(0xffffffffu, bad, 0);
  if (FULL) {
    // L^{-1}[j][k] at k NC + j: (m,c | n,c') = delta_cc' K^{-1}[m][n] + w(m,c) w(n,c') / s,
    // (m,c | p) = -w(m,c) / s, (p | n,c') = -w(n,c') / s, (p | p) = 1 / s
    double* o = out + p * (int64_t)NC * NC;
    for (int e = lane; e < NC * NC; e += 32) {
      const int k = e / NC, j = e % NC;
      double val;
      if (j == NC - 1 && k == NC - 1) val = sinv;
      else if (j == NC - 1) val = -Z[(NE + k % D) * NV + k / D] * sinv;
      else if (k == NC - 1) val = -Z[(NE + j % D) * NV + j / D] * sinv;
      else
        val = (j % D == k % D ? Z[(j / D) * NV + k / D] : 0.0) +
              Z[(NE + j % D) * NV + j / D] * Z[(NE + k % D) * NV + k / D] * sinv;
      o[e] = val;
    }
  } else {
    for (int k = lane; k < NF; k += 32) {
      double val;
      if (k < NV) val = Z[k];
      else if (k < NV + NV * D) {
        const int m = (k - NV) / D, c = (k - NV) % D;
        val = Z[(1 + c) * NV + m];
      } else val = sinv;
      out[k * np + p] = val;
    }
  }
  if (bad && lane == 0) atomicExch(err, 1);
}

// Global DoF of Q1-Q1 box position k (velocity m d + c, pressure NC - 1) of the
// subdomain at vertex v, -1 if not in it.
template <int D>
__device__ __forceinline__ int64_t q1_box_dof(const Geo& g, const int* v, int64_t p, int k) {
  constexpr int NC = Q1Box<D>::NC;
  if (k == NC - 1) return g.n_u + p;
  const int m = k / D;
  if (!q1_free<D>(g, v, m)) return -1;
  int a[3];
  q1_tuple(m, a);
  int64_t id = 0;
  for (int d = D - 1; d >= 0; --d) id = id * (g.N + 1) + (v[d] - 1 + a[d]);
  return D * id + k % D;
}
template <int D>
__device__ void q1_warp_full_solve(const double* __restrict__ Inv, const double* rloc, double* y) {
  constexpr int NC = Q1Box<D>::NC;
  const int lane = threadIdx.x & 31;
  for (int j = lane; j < NC; j += 32) {
    double s = 0.0;
    for (int k = 0; k < NC; ++k) s += Inv[(int64_t)k * NC + j] * rloc[k];
    y[j] = s;
  }
  __syncwarp();
}

// AV (Eq. 12) on Q1-Q1, step 1: corr[p][k] = omega_p (L_p^{-1} r_p)_k, one warp per subdomain.
template <int D>
__global__ void k_av_q1_corr(Geo g, const double* __restrict__ inv, const double* __restrict__ omega,
                             const double* __restrict__ r, double* __restrict__ corr) {
  constexpr int NC = Q1Box<D>::NC;
  constexpr int WPB = 4;
  __shared__ double rl[WPB][NC], yl[WPB][NC];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = blockIdx.x * (int64_t)WPB + wi;
  if (p >= g.n_p) return;
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  for (int k = lane; k < NC; k += 32) {
    const int64_t dof = q1_box_dof<D>(g, v, p, k);
    rl[wi][k] = dof >= 0 ? r[dof] : 0.0;
  }
  __syncwarp();
  q1_warp_full_solve<D>(inv + p * (int64_t)NC * NC, rl[wi], yl[wi]);
  const double om = omega[p];
  for (int k = lane; k < NC; k += 32) corr[p * NC + k] = om * yl[wi][k];
}

// AV on Q1-Q1, step 2: x[dof] += sum over the subdomains containing dof (ascending) of corr.
template <int D>
__global__ void k_av_q1_gather(Geo g, const double* __restrict__ corr, double* __restrict__ x) {
  constexpr int NC = Q1Box<D>::NC;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  if (i >= g.n_u) {
    x[i] += corr[(i - g.n_u) * NC + NC - 1];
    return;
  }
  int64_t I[3] = {0, 0, 0};
  int c;
  vel_node(g, i, I, c);
  if (node_on_boundary(g, I)) return;
  double s = 0.0;
  for (int v2 = (D == 3 ? (int)I[2] - 1 : 0); v2 <= (D == 3 ? (int)I[2] + 1 : 0); ++v2)
    for (int v1 = (int)I[1] - 1; v1 <= (int)I[1] + 1; ++v1)
      for (int v0 = (int)I[0] - 1; v0 <= (int)I[0] + 1; ++v0) {
        const int vv[3] = {v0, v1, v2};
        int64_t p = 0;
        int m = 0;
        for (int d = D - 1; d >= 0; --d) {
          p = p * (g.N + 1) + vv[d];
          m = m * 3 + (int)(I[d] - vv[d] + 1);
        }
        s += corr[p * NC + m * D + c];  // free I: every v in [I-1, I+1] is a vertex
      }
  x[i] += s;
}

// MV (Eq. 11 with the residual refresh of Eq. 15) on Q1-Q1 over one colour
// class (vertices equal mod 4 on every axis): a subdomain writes vertices
// v-1..v+1 and its refresh reads v-2..v+2, so subdomains of a class four
// vertices apart neither overlap nor read each other's writes.
template <int D>
__global__ void k_mv_q1_colour(Geo g, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const double* __restrict__ va, const double* __restrict__ inv,
                               const double* __restrict__ omega, const double* __restrict__ b,
                               double* __restrict__ x, int colour) {
  constexpr int NC = Q1Box<D>::NC;
  constexpr int WPB = 4;
  __shared__ double rl[WPB][NC], yl[WPB][NC];
  __shared__ int64_t dl[WPB][NC];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int col[3] = {colour & 3, (colour >> 2) & 3, (colour >> 4) & 3};
  int cnt[3] = {1, 1, 1};
  int64_t tot = 1;
  for (int d = 0; d < D; ++d) {
    cnt[d] = col[d] <= g.N ? (g.N - col[d]) / 4 + 1 : 0;
    tot *= cnt[d];
  }
  const int64_t t = blockIdx.x * (int64_t)WPB + wi;
  if (t >= tot) return;
  int v[3] = {0, 0, 0};
  {
    int64_t tt = t;
    for (int d = 0; d < D; ++d) { v[d] = col[d] + 4 * (int)(tt % cnt[d]); tt /= cnt[d]; }
  }
  int64_t p = 0;
  for (int d = D - 1; d >= 0; --d) p = p * (g.N + 1) + v[d];
  for (int k = lane; k < NC; k += 32) {
    const int64_t dof = q1_box_dof<D>(g, v, p, k);
    dl[wi][k] = dof;
    double s = 0.0;
    if (dof >= 0) {
      s = b[dof];
      for (int64_t q = rp[dof]; q < rp[dof + 1]; ++q) s -= va[q] * x[ci[q]];
    }
    rl[wi][k] = s;
  }
  __syncwarp();
  q1_warp_full_solve<D>(inv + p * (int64_t)NC * NC, rl[wi], yl[wi]);
  const double om = omega[p];
  for (int k = lane; k < NC; k += 32)
    if (dl[wi][k] >= 0) x[dl[wi][k]] += om * yl[wi][k];
}

// Full inverses (AV/MV) on Q1-Q1 expanded to the compact sorted order.
template <int D>
__global__ void k_export_q1_full(Geo g, const double* __restrict__ inv, int64_t first, int64_t count,
                                 double* __restrict__ out) {
  constexpr int NC = Q1Box<D>::NC;
  __shared__ int colmap[NC];
  __shared__ int ncol;
  const int64_t p = first + blockIdx.x;
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  if (threadIdx.x == 0) {
    int c = 0;
    for (int k = 0; k < NC; ++k)
      if (q1_box_dof<D>(g, v, p, k) >= 0) colmap[c++] = k;
    ncol = c;
  }
  __syncthreads();
  double* o = out + blockIdx.x * (int64_t)NC * NC;
  for (int e = threadIdx.x; e < NC * NC; e += blockDim.x) {
    const int jr = e / NC, kc = e % NC;
    double val = 0.0;
    if (jr < ncol && kc < ncol) val = inv[p * (int64_t)NC * NC + (int64_t)colmap[kc] * NC + colmap[jr]];
    o[e] = val;
  }
}

template <typename T>
__global__ void k_q1_pack(const double* __restrict__ stage, int64_t n, T* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = Fmt<T>::enc(stage[i]);
}

// Owned row j of L_i^{-1} at box position k (velocity m d + c, pressure NC - 1)
// from the factored values of subdomain p (stage: SoA, NF x np, fp64):
//   row c < d (vertex i's component c): delta_{c, k%d} K^{-1}[CEN, k/d] + w(CEN,c) w(k) / s,
//                                       -w(CEN,c) / s at the pressure;
//   row d (p_i): -w(k) / s, 1 / s at the pressure.
template <int D>
__device__ __forceinline__ double q1_row_entry(const double* __restrict__ stage, int64_t np, int64_t p, int j,
                                               int k) {
  using B = Q1Box<D>;
  constexpr int NV = B::NV, NC = B::NC, NF = B::NF;
  const double sig = stage[(int64_t)(NF - 1) * np + p];
  if (j == D) return k == NC - 1 ? sig : -stage[(int64_t)(NV + k) * np + p] * sig;
  const double wj = stage[(int64_t)(NV + B::CEN * D + j) * np + p];
  if (k == NC - 1) return -wj * sig;
  return (k % D == j ? stage[(int64_t)(k / D) * np + p] : 0.0) + wj * stage[(int64_t)(NV + k) * np + p] * sig;
}

// Q1-Q1 dense-row storage (the owned rows of Sec. 4.3): the d + 1 owned rows
// over the NC box positions rounded into T (fp8 with an fp32 scale
// max|row| / 448 per row); element (j, k) of subdomain p at (j NC + k) np + p,
// the scale of row j at j np + p.  One thread per (row, subdomain).
template <int D, typename T>
__global__ void k_q1_rows(const double* __restrict__ stage, int64_t np, T* __restrict__ out,
                          float* __restrict__ scale) {
  using B = Q1Box<D>;
  constexpr int NC = B::NC, NR = B::NR;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= np * NR) return;
  const int j = (int)(t / np);
  const int64_t p = t - j * np;
  double sc = 1.0;
  if (Fmt<T>::scaled) {
    double m = 0.0;
    for (int k = 0; k < NC; ++k) m = fmax(m, fabs(q1_row_entry<D>(stage, np, p, j, k)));
    sc = m == 0.0 ? 1.0 : (double)(float)(m / 448.0);
    scale[(int64_t)j * np + p] = (float)sc;
  }
  for (int k = 0; k < NC; ++k)
    out[((int64_t)j * NC + k) * np + p] = Fmt<T>::enc(q1_row_entry<D>(stage, np, p, j, k) / sc);
}

// RAV step on Q1-Q1 with dense rows, one thread per subdomain: y_j = sum_k
// row_j[k] r[k] over the box (fp64, or fp32 on the fp32 residual for reduced
// formats, times the row scale), x[owned j] += omega y_j.
template <int D, typename T>
__global__ void __launch_bounds__(128) k_rav_apply_q1_rows(Geo g, const T* __restrict__ st,
                                                           const float* __restrict__ scale,
                                                           const double* __restrict__ omega,
                                                           const AccT<T>* __restrict__ r, double* __restrict__ x,
                                                           int64_t np) {
  using B = Q1Box<D>;
  using A = AccT<T>;
  constexpr int NC = B::NC, NR = B::NR;
  __shared__ float lut[256];
  if (Fmt<T>::scaled) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
      __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)i, __NV_E4M3);
      lut[i] = __half2float(__half(h));
    }
    __syncthreads();
  }
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  const int N = g.N;
  const int64_t N1 = N + 1;
  A y[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) y[j] = 0;
#pragma unroll
  for (int a2 = 0; a2 < (D == 3 ? 3 : 1); ++a2) {
    const int J2 = D == 3 ? v[2] - 1 + a2 : 0;
    const bool ok2 = D == 2 || (J2 >= 1 && J2 <= N - 1);
#pragma unroll
    for (int a1 = 0; a1 < 3; ++a1) {
      const int J1 = v[1] - 1 + a1;
      const bool ok1 = ok2 && J1 >= 1 && J1 <= N - 1;
#pragma unroll
      for (int a0 = 0; a0 < 3; ++a0) {
        const int n = a0 + 3 * a1 + 9 * a2;
        const int J0 = v[0] - 1 + a0;
        const bool ok = ok1 && J0 >= 1 && J0 <= N - 1;
        const int64_t base = (int64_t)D * (J0 + N1 * (J1 + N1 * J2));
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const A rv = ok ? r[base + c] : (A)0;
#pragma unroll
          for (int j = 0; j < NR; ++j)
            y[j] += (A)Fmt<T>::dec(ld_stream(st + ((int64_t)j * NC + n * D + c) * np + p), lut) * rv;
        }
      }
    }
  }
  const A rp = r[g.n_u + p];
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    y[j] += (A)Fmt<T>::dec(ld_stream(st + ((int64_t)j * NC + NC - 1) * np + p), lut) * rp;
    if (Fmt<T>::scaled) y[j] *= (A)scale[(int64_t)j * np + p];
  }
  const double om = omega[p];
  bool cfree = true;
#pragma unroll
  for (int d = 0; d < D; ++d) cfree &= v[d] >= 1 && v[d] <= N - 1;
  if (cfree) {
#pragma unroll
    for (int c = 0; c < D; ++c) x[D * p + c] += om * (double)y[c];
  }
  x[g.n_u + p] += om * (double)y[D];
}

// Dense Q1-Q1 rows expanded (scale applied) to the compact sorted order.
template <int D, typename T>
__global__ void k_export_q1_rows(Geo g, const T* __restrict__ st, const float* __restrict__ scale, int64_t np,
                                 int64_t first, int64_t count, double* __restrict__ out) {
  using B = Q1Box<D>;
  constexpr int NC = B::NC, NR = B::NR;
  __shared__ float lut[256];
  __shared__ int colmap[NC], rowmap[NR];
  __shared__ int ncol, nrow;
  if (Fmt<T>::scaled) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
      __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)i, __NV_E4M3);
      lut[i] = __half2float(__half(h));
    }
  }
  const int64_t p = first + blockIdx.x;
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  if (threadIdx.x == 0) {
    int c = 0;
    for (int m = 0; m < B::NV; ++m)
      if (q1_free<D>(g, v, m))
        for (int cc = 0; cc < D; ++cc) colmap[c++] = m * D + cc;
    colmap[c++] = NC - 1;
    ncol = c;
    int rr = 0;
    if (q1_free<D>(g, v, B::CEN))
      for (int cc = 0; cc < D; ++cc) rowmap[rr++] = cc;
    rowmap[rr++] = NR - 1;
    nrow = rr;
  }
  __syncthreads();
  double* o = out + blockIdx.x * (int64_t)NR * NC;
  for (int e = threadIdx.x; e < NR * NC; e += blockDim.x) {
    const int jr = e / NC, kc = e % NC;
    double val = 0.0;
    if (jr < nrow && kc < ncol) {
      const int j = rowmap[jr], k = colmap[kc];
      val = (double)Fmt<T>::dec(st[((int64_t)j * NC + k) * np + p], lut);
      if (Fmt<T>::scaled) val *= (double)scale[(int64_t)j * np + p];
    }
    o[e] = val;
  }
}

// RAV step on Q1-Q1 (Eq. 13), one thread per subdomain: with r_u, r_p the
// residual on the box, t = (w^T r_u - r_p) / s,
//   x[v, c] += omega (sum_m K^{-1}[CEN, m] r_u[m, c] + w[CEN, c] t)   (v free)
//   x[p_i]  += omega (-t).
// Stored values in T, accumulation in fp64 (T = double, r fp64) or fp32
// (reduced formats, r the fp32 copy); x is updated in fp64.
template <int D, typename T>
__global__ void __launch_bounds__(128) k_rav_apply_q1(Geo g, const T* __restrict__ st,
                                                      const double* __restrict__ omega,
                                                      const AccT<T>* __restrict__ r, double* __restrict__ x,
                                                      int64_t np) {
  using B = Q1Box<D>;
  using A = AccT<T>;
  constexpr int NV = B::NV, NF = B::NF;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= np) return;
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  const int N = g.N;
  const int64_t N1 = N + 1;
  A y[D], wc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) y[c] = wc[c] = 0;
  A t = 0;
#pragma unroll
  for (int a2 = 0; a2 < (D == 3 ? 3 : 1); ++a2) {
    const int J2 = D == 3 ? v[2] - 1 + a2 : 0;
    const bool ok2 = D == 2 || (J2 >= 1 && J2 <= N - 1);
#pragma unroll
    for (int a1 = 0; a1 < 3; ++a1) {
      const int J1 = v[1] - 1 + a1;
      const bool ok1 = ok2 && J1 >= 1 && J1 <= N - 1;
#pragma unroll
      for (int a0 = 0; a0 < 3; ++a0) {
        const int n = a0 + 3 * a1 + 9 * a2;
        const int J0 = v[0] - 1 + a0;
        const bool ok = ok1 && J0 >= 1 && J0 <= N - 1;
        const int64_t base = (int64_t)D * (J0 + N1 * (J1 + N1 * J2));
        A ru[D];
        if constexpr (D == 2 && std::is_same<A, float>::value) {
          float2 rv = make_float2(0.f, 0.f);
          if (ok) rv = *reinterpret_cast<const float2*>(r + base);
          ru[0] = rv.x;
          ru[1] = rv.y;
        } else {
#pragma unroll
          for (int c = 0; c < D; ++c) ru[c] = ok ? r[base + c] : (A)0;
        }
        const A kq = (A)Fmt<T>::dec(ld_stream(st + n * np + p), nullptr);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const A wv = (A)Fmt<T>::dec(ld_stream(st + (NV + n * D + c) * np + p), nullptr);
          y[c] += kq * ru[c];
          t += wv * ru[c];
          if (n == B::CEN) wc[c] = wv;
        }
      }
    }
  }
  const A tau = (A)Fmt<T>::dec(ld_stream(st + (NF - 1) * np + p), nullptr) * (t - r[g.n_u + p]);
  const double om = omega[p];
  bool cfree = true;
#pragma unroll
  for (int d = 0; d < D; ++d) cfree &= v[d] >= 1 && v[d] <= N - 1;
  if (cfree) {
#pragma unroll
    for (int c = 0; c < D; ++c) x[D * p + c] += om * (double)(y[c] + wc[c] * tau);
  }
  x[g.n_u + p] -= om * (double)tau;
}

// Inspection on Q1-Q1: subdomain sizes, sorted DoF lists, and the owned rows
// of L_i^{-1} rebuilt from the stored values,
//   (CEN,c | n,c') = delta_cc' K^{-1}[CEN,n] + w(CEN,c) w(n,c') / s,  (CEN,c | p) = -w(CEN,c) / s,
//   (p | n,c') = -w(n,c') / s,  (p | p) = 1 / s,
// padded to NR x NC per subdomain.
template <int D>
__global__ void k_q1_patch_count(Geo g, int32_t* __restrict__ cnt) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= g.n_p) return;
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  int c = 1;
  for (int m = 0; m < Q1Box<D>::NV; ++m) c += q1_free<D>(g, v, m) ? D : 0;
  cnt[p] = c;
}
template <int D>
__global__ void k_q1_patch_list(Geo g, const int32_t* __restrict__ off, int32_t* __restrict__ dofs) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= g.n_p) return;
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  int32_t pos = off[p];
  for (int m = 0; m < Q1Box<D>::NV; ++m) {
    if (!q1_free<D>(g, v, m)) continue;
    int a[3];
    q1_tuple(m, a);
    int64_t id = 0;
    for (int d = D - 1; d >= 0; --d) id = id * (g.N + 1) + (v[d] - 1 + a[d]);
    for (int c = 0; c < D; ++c) dofs[pos++] = (int32_t)(D * id + c);
  }
  dofs[pos] = (int32_t)(g.n_u + p);
}
template <int D, typename T>
__global__ void k_export_q1(Geo g, const T* __restrict__ st, int64_t np, int64_t first, int64_t count,
                            double* __restrict__ out) {
  using B = Q1Box<D>;
  constexpr int NV = B::NV, NC = B::NC, NR = B::NR, NF = B::NF;
  __shared__ int colmap[NC], rowmap[NR];
  __shared__ int ncol, nrow;
  const int64_t p = first + blockIdx.x;
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  if (threadIdx.x == 0) {
    int c = 0;
    for (int m = 0; m < NV; ++m)
      if (q1_free<D>(g, v, m))
        for (int cc = 0; cc < D; ++cc) colmap[c++] = m * D + cc;
    colmap[c++] = NC - 1;
    ncol = c;
    int rr = 0;
    if (q1_free<D>(g, v, B::CEN))
      for (int cc = 0; cc < D; ++cc) rowmap[rr++] = cc;
    rowmap[rr++] = NR - 1;
    nrow = rr;
  }
  __syncthreads();
  auto val_at = [&](int k) { return (double)Fmt<T>::dec(st[k * np + p], nullptr); };
  const double sig = val_at(NF - 1);
  double* o = out + blockIdx.x * (int64_t)NR * NC;
  for (int e = threadIdx.x; e < NR * NC; e += blockDim.x) {
    const int jr = e / NC, kc = e % NC;
    double val = 0.0;
    if (jr < nrow && kc < ncol) {
      const int j = rowmap[jr], k = colmap[kc];
      const bool prow = j == NR - 1, pcol = k == NC - 1;
      if (prow && pcol) val = sig;
      else if (prow) val = -val_at(NV + k) * sig;
      else {
        const double wm = val_at(NV + B::CEN * D + j);
        if (pcol) val = -wm * sig;
        else val = (k % D == j ? val_at(k / D) : 0.0) + wm * val_at(NV + k) * sig;
      }
    }
    o[e] = val;
  }
}

__global__ void k_fill(double* __restrict__ a, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}
__global__ void k_f64_to_f32(const double* __restrict__ a, int64_t n, float* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_f32_to_f64(const float* __restrict__ a, int64_t n, double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

}  // namespace rav

using namespace rav;

static size_t elem_size(int prec) {
  switch (prec) {
    case RAV_F64:
    case RAV_F64_ROWS: return 8;
    case RAV_F32:
    case RAV_F32_FACT: return 4;
    case RAV_BF16:
    case RAV_BF16_FACT: return 2;
    default: return 1;
  }
}
static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}
static bool factored_prec(int prec) { return prec == RAV_F64 || prec == RAV_F32_FACT || prec == RAV_BF16_FACT; }

template <int D>
static int setup_level(rav_smoother* sm, int l, cudaStream_t s, int* err_dev) {
  using B = BoxT<D>;
  rav_mg* mg = sm->mg;
  const Level& L = mg->lev[l];
  SmLevel& S_ = sm->lev[l];
  const Geo& g = L.g;
  S_.np = g.n_p;
  const bool all = sm->kind != RAV_RAV;
  const bool fact = sm->kind == RAV_RAV && factored_prec(sm->prec);
  S_.factored = fact;
  const int NROW = all ? B::NC : B::NR;
  const int64_t per = fact ? B::NF : (int64_t)NROW * B::NC;  // staging doubles per subdomain
  RAV_CUDA(cudaMalloc(&S_.omega, sizeof(double) * S_.np));
  k_fill<<<grid_for(S_.np, 256), 256, 0, s>>>(S_.omega, S_.np, sm->omega);
  if (sm->kind == RAV_RAV && sm->prec != RAV_F64 && sm->prec != RAV_F64_ROWS)
    RAV_CUDA(cudaMalloc(&S_.r32, sizeof(float) * g.n));
  if (all) {
    RAV_CUDA(cudaMalloc(&S_.inv, sizeof(double) * S_.np * B::NC * B::NC));
    if (sm->kind == RAV_AV) RAV_CUDA(cudaMalloc(&S_.corr, sizeof(double) * S_.np * B::NC));
  } else if (fact) {
    S_.units = S_.np * B::NON;
    S_.split = 1;  // packed for one thread per owned node; vanka_setup tunes it afterwards
    const int64_t groups = (S_.units + 31) / 32;
    const size_t es = elem_size(sm->prec);
    RAV_CUDA(cudaMalloc(&S_.inv, es * groups * 32 * B::NV));
    RAV_CUDA(cudaMemsetAsync(S_.inv, 0, es * groups * 32 * B::NV, s));
    RAV_CUDA(cudaMalloc(&S_.ws, es * S_.np * (D * B::NV + 1)));
  } else {
    S_.units = S_.np * B::NCH;
    const int64_t groups = (S_.units + 31) / 32;
    RAV_CUDA(cudaMalloc(&S_.inv, elem_size(sm->prec) * groups * 32 * B::NC * B::RB));
    RAV_CUDA(cudaMemsetAsync(S_.inv, 0, elem_size(sm->prec) * groups * 32 * B::NC * B::RB, s));
    if (sm->prec == RAV_FP8) RAV_CUDA(cudaMalloc(&S_.scale, sizeof(float) * groups * 32 * B::RB));
  }
  // factorise in batches; staging rows in fp64
  const int64_t batch = std::min<int64_t>(S_.np, all ? 8192 : 32768);
  double* stage = nullptr;
  RAV_CUDA(cudaMallocAsync(&stage, sizeof(double) * batch * per, s));
  // the staging buffer is released on every exit path below
  struct StageFree {
    double* p;
    cudaStream_t s;
    ~StageFree() { cudaFreeAsync(p, s); }
  } stage_free{stage, s};
  const size_t smem = sizeof(double) * (B::NV * B::NV + 2 * B::NV * D + 32 * B::NV);
  auto kf = all ? k_factor<D, 1> : (fact ? k_factor<D, 2> : k_factor<D, 0>);
  RAV_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int threads = D == 2 ? 128 : 256;
  for (int64_t f = 0; f < S_.np; f += batch) {
    const int64_t cnt = std::min<int64_t>(batch, S_.np - f);
    kf<<<(unsigned)cnt, threads, smem, s>>>(g, L.rp, L.va, f, cnt, stage, err_dev);
    if (fact) {
      const int64_t tot = cnt * (D * B::NV + 1);
      const unsigned gb = (unsigned)((tot + 127) / 128);
      const int lg = 5 - ilog2(S_.split);
      if (sm->prec == RAV_F64)
        k_pack_fact<D, double><<<gb, 128, 0, s>>>(stage, f, cnt, (double*)S_.inv, (double*)S_.ws, lg);
      else if (sm->prec == RAV_F32_FACT)
        k_pack_fact<D, float><<<gb, 128, 0, s>>>(stage, f, cnt, (float*)S_.inv, (float*)S_.ws, lg);
      else
        k_pack_fact<D, __nv_bfloat16>
            <<<gb, 128, 0, s>>>(stage, f, cnt, (__nv_bfloat16*)S_.inv, (__nv_bfloat16*)S_.ws, lg);
    } else if (all) {
      const int64_t tot = cnt * B::NC * B::NC;
      k_pack_full<D><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(stage, f, cnt, (double*)S_.inv);
    } else {
      const int64_t tot = cnt * B::NR;
      const unsigned gb = (unsigned)((tot + 127) / 128);
      switch (sm->prec) {
        case RAV_F64_ROWS:
          k_pack_rav<D, double><<<gb, 128, 0, s>>>(stage, f, cnt, (double*)S_.inv, S_.scale);
          break;
        case RAV_F32: k_pack_rav<D, float><<<gb, 128, 0, s>>>(stage, f, cnt, (float*)S_.inv, S_.scale); break;
        case RAV_BF16:
          k_pack_rav<D, __nv_bfloat16><<<gb, 128, 0, s>>>(stage, f, cnt, (__nv_bfloat16*)S_.inv, S_.scale);
          break;
        default: k_pack_rav<D, fp8_t><<<gb, 128, 0, s>>>(stage, f, cnt, (fp8_t*)S_.inv, S_.scale); break;
      }
    }
    RAV_CUDA(cudaGetLastError());
  }
  return RAV_OK;
}

// Q1-Q1 level: RAV with factored storage (RAV_F64 / RAV_F32_FACT /
// RAV_BF16_FACT) or the owned rows (RAV_F64_ROWS / RAV_F32 / RAV_BF16 /
// RAV_FP8), one thread per subdomain, no split; AV and MV with the full fp64
// inverse per subdomain.
template <int D>
static int setup_level_q1(rav_smoother* sm, int l, cudaStream_t s, int* err_dev) {
  using B = Q1Box<D>;
  const Level& L = sm->mg->lev[l];
  SmLevel& S_ = sm->lev[l];
  const Geo& g = L.g;
  S_.np = g.n_p;
  S_.units = g.n_p;
  S_.split = 1;
  RAV_CUDA(cudaMalloc(&S_.omega, sizeof(double) * S_.np));
  k_fill<<<grid_for(S_.np, 256), 256, 0, s>>>(S_.omega, S_.np, sm->omega);
  if (sm->kind != RAV_RAV) {
    S_.factored = false;
    RAV_CUDA(cudaMalloc(&S_.inv, sizeof(double) * S_.np * B::NC * B::NC));
    if (sm->kind == RAV_AV) RAV_CUDA(cudaMalloc(&S_.corr, sizeof(double) * S_.np * B::NC));
    constexpr int wpb = D == 3 ? 2 : 4;
    k_factor_q1<D, true><<<(unsigned)((S_.np + wpb - 1) / wpb), 32 * wpb, 0, s>>>(g, L.rp, L.va, S_.np,
                                                                                (double*)S_.inv, err_dev);
    RAV_CUDA(cudaGetLastError());
    return RAV_OK;
  }
  if (!factored_prec(sm->prec)) {
    S_.factored = false;
    const int64_t nrow = S_.np * B::NR;
    RAV_CUDA(cudaMalloc(&S_.inv, elem_size(sm->prec) * nrow * B::NC));
    if (sm->prec == RAV_FP8) RAV_CUDA(cudaMalloc(&S_.scale, sizeof(float) * nrow));
    if (sm->prec != RAV_F64_ROWS) RAV_CUDA(cudaMalloc(&S_.r32, sizeof(float) * g.n));
    double* stage = nullptr;
    RAV_CUDA(cudaMallocAsync(&stage, sizeof(double) * S_.np * B::NF, s));
    k_factor_q1<D, false><<<(unsigned)((S_.np + 3) / 4), 128, 0, s>>>(g, L.rp, L.va, S_.np, stage, err_dev);
    const unsigned gr = (unsigned)((nrow + 127) / 128);
    switch (sm->prec) {
      case RAV_F64_ROWS: k_q1_rows<D, double><<<gr, 128, 0, s>>>(stage, S_.np, (double*)S_.inv, S_.scale); break;
      case RAV_F32: k_q1_rows<D, float><<<gr, 128, 0, s>>>(stage, S_.np, (float*)S_.inv, S_.scale); break;
      case RAV_BF16:
        k_q1_rows<D, __nv_bfloat16><<<gr, 128, 0, s>>>(stage, S_.np, (__nv_bfloat16*)S_.inv, S_.scale);
        break;
      default: k_q1_rows<D, fp8_t><<<gr, 128, 0, s>>>(stage, S_.np, (fp8_t*)S_.inv, S_.scale); break;
    }
    cudaFreeAsync(stage, s);
    RAV_CUDA(cudaGetLastError());
    return RAV_OK;
  }
  S_.factored = true;
  const int64_t tot = S_.np * B::NF;
  RAV_CUDA(cudaMalloc(&S_.inv, elem_size(sm->prec) * tot));
  const unsigned gf = (unsigned)((S_.np + 3) / 4);
  if (sm->prec == RAV_F64) {
    k_factor_q1<D, false><<<gf, 128, 0, s>>>(g, L.rp, L.va, S_.np, (double*)S_.inv, err_dev);
  } else {
    RAV_CUDA(cudaMalloc(&S_.r32, sizeof(float) * g.n));
    double* stage = nullptr;
    RAV_CUDA(cudaMallocAsync(&stage, sizeof(double) * tot, s));
    k_factor_q1<D, false><<<gf, 128, 0, s>>>(g, L.rp, L.va, S_.np, stage, err_dev);
    const unsigned gp = (unsigned)((tot + 255) / 256);
    if (sm->prec == RAV_F32_FACT) k_q1_pack<float><<<gp, 256, 0, s>>>(stage, tot, (float*)S_.inv);
    else k_q1_pack<__nv_bfloat16><<<gp, 256, 0, s>>>(stage, tot, (__nv_bfloat16*)S_.inv);
    cudaFreeAsync(stage, s);
  }
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

static int tune_apply_split(rav_smoother* sm, cudaStream_t s);

extern "C" int vanka_setup(rav_mg* mg, int kind, int precision, double omega, rav_stream stream,
                           rav_smoother** out) {
  if (!mg || !out || (kind != RAV_RAV && kind != RAV_AV && kind != RAV_MV_COLOURED)) return RAV_ERR_ARG;
  if (precision < RAV_F64 || precision > RAV_BF16_FACT) return RAV_ERR_ARG;
  if (kind != RAV_RAV && precision != RAV_F64 && precision != RAV_F64_ROWS) return RAV_ERR_ARG;
  const bool q1 = mg->elem == RAV_ELEM_Q1Q1;
  cudaStream_t s = S(stream);
  *out = nullptr;
  rav_smoother* sm = new rav_smoother();
  sm->mg = mg;
  sm->kind = kind;
  sm->prec = precision;
  sm->omega = omega;
  int* err_dev = nullptr;
  int rc = RAV_OK;
  if (cudaMalloc(&err_dev, sizeof(int)) != cudaSuccess) { delete sm; return RAV_ERR_CUDA; }
  cudaMemsetAsync(err_dev, 0, sizeof(int), s);
  for (int l = 1; l < mg->nlev && rc == RAV_OK; ++l) {
    if (q1) rc = mg->dim == 2 ? setup_level_q1<2>(sm, l, s, err_dev) : setup_level_q1<3>(sm, l, s, err_dev);
    else rc = mg->dim == 2 ? setup_level<2>(sm, l, s, err_dev) : setup_level<3>(sm, l, s, err_dev);
  }
  int err = 0;
  if (rc == RAV_OK) {
    if (cudaMemcpyAsync(&err, err_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = RAV_ERR_CUDA;
    else if (err)
      rc = RAV_ERR_SINGULAR_PATCH;
  }
  cudaFree(err_dev);
  if (rc == RAV_OK && !q1) rc = tune_apply_split(sm, s);
  if (rc == RAV_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = RAV_ERR_CUDA;
  if (rc != RAV_OK) {
    vanka_destroy(sm);
    return rc;
  }
  *out = sm;
  return RAV_OK;
}

extern "C" void vanka_destroy(rav_smoother* sm) {
  if (!sm) return;
  cudaDeviceSynchronize();
  if (sm->mg) drop_graphs(sm->mg, sm);
  for (int l = 0; l < kMaxLevels; ++l) {
    cudaFree(sm->lev[l].inv);
    cudaFree(sm->lev[l].ws);
    cudaFree(sm->lev[l].scale);
    cudaFree(sm->lev[l].r32);
    cudaFree(sm->lev[l].omega);
    cudaFree(sm->lev[l].corr);
    cudaFree(sm->lev[l].lsum);
    cudaFree(sm->lev[l].lcnt);
    cudaFree(sm->lev[l].ones);
    cudaFree(sm->lev[l].ctmp);
    cudaFree(sm->lev[l].stmp);
    cudaFree(sm->lev[l].rtmp);
    cudaFree(sm->lev[l].xalt);
    staged_free(sm->lev[l]);
  }
  delete sm;
}

static int regroup(rav_smoother* sm, int level, int split, cudaStream_t s) {
  SmLevel& SL = sm->lev[level];
  const int NV = sm->mg->dim == 2 ? 25 : 125;
  if (split == SL.split) return RAV_OK;
  const size_t es = elem_size(sm->prec);
  const size_t bytes = es * ((SL.units + 31) / 32) * 32 * NV;
  void* dst = nullptr;
  RAV_CUDA(cudaMalloc(&dst, bytes));
  RAV_CUDA(cudaMemsetAsync(dst, 0, bytes, s));
  const int ls = 5 - ilog2(SL.split), ld = 5 - ilog2(split);
  const unsigned gb = (unsigned)((SL.units * NV + 255) / 256);
  if (es == 8) k_regroup<double><<<gb, 256, 0, s>>>((const double*)SL.inv, (double*)dst, SL.units, NV, ls, ld);
  else if (es == 4) k_regroup<float><<<gb, 256, 0, s>>>((const float*)SL.inv, (float*)dst, SL.units, NV, ls, ld);
  else k_regroup<uint16_t><<<gb, 256, 0, s>>>((const uint16_t*)SL.inv, (uint16_t*)dst, SL.units, NV, ls, ld);
  RAV_CUDA(cudaGetLastError());
  RAV_CUDA(cudaStreamSynchronize(s));
  cudaFree(SL.inv);
  SL.inv = dst;
  SL.split = split;
  return RAV_OK;
}

// Threads per owned node of the factored apply, per level: each candidate is
// timed over 5 applies on the level's work vectors (zeroed first and after),
// and the fewest threads within 3 % of the fastest win.
static int tune_apply_split(rav_smoother* sm, cudaStream_t s) {
  rav_mg* mg = sm->mg;
  const int maxs = mg->dim == 2 ? 8 : 4;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RAV_CUDA(cudaEventCreate(&e0));
  RAV_CUDA(cudaEventCreate(&e1));
  int rc = RAV_OK;
  for (int l = 1; l < mg->nlev && rc == RAV_OK; ++l) {
    SmLevel& SL = sm->lev[l];
    Level& L = mg->lev[l];
    if (!SL.factored) continue;
    cudaMemsetAsync(L.r, 0, sizeof(double) * L.g.n, s);
    if (SL.r32) cudaMemsetAsync(SL.r32, 0, sizeof(float) * L.g.n, s);
    float t[4] = {0, 0, 0, 0};
    int nc = 0;
    for (int sp = 1; sp <= maxs && rc == RAV_OK; sp *= 2, ++nc) {
      rc = regroup(sm, l, sp, s);
      for (int w = 0; w < 2 && rc == RAV_OK; ++w) rc = apply_with_omega(sm, l, L.r, L.x, SL.omega, s, SL.r32);
      cudaEventRecord(e0, s);
      for (int w = 0; w < 5 && rc == RAV_OK; ++w) rc = apply_with_omega(sm, l, L.r, L.x, SL.omega, s, SL.r32);
      cudaEventRecord(e1, s);
      if (rc == RAV_OK &&
          (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[nc], e0, e1) != cudaSuccess))
        rc = RAV_ERR_CUDA;
    }
    if (rc != RAV_OK) break;
    float best = t[0];
    for (int i = 1; i < nc; ++i) best = t[i] < best ? t[i] : best;
    int pick = 0;
    while (t[pick] > 1.03f * best) ++pick;
    rc = regroup(sm, l, 1 << pick, s);
    // reduced storage: the staged kernel (shared-memory residual tiles,
    // streamed chunks) replaces the grouped one where it is 3 % faster
    if (rc == RAV_OK && sm->prec != RAV_F64) {
      const int splits[3] = {1, 2, 4};
      const int nsplit = mg->dim == 2 ? 2 : 3;
      float tb = 0.97f * best;
      int sbest = 0, cbest = 0;
      for (int ci = 0; ci < nsplit && rc == RAV_OK; ++ci)
        for (int tc = 0; tc < 3 && rc == RAV_OK; ++tc) {  // the three best tilings
          const int rb = staged_build(sm, l, splits[ci], s, tc);
          if (rb == RAV_ERR_ARG) break;  // no further candidate
          rc = rb;
          for (int w = 0; w < 2 && rc == RAV_OK; ++w) rc = apply_with_omega(sm, l, L.r, L.x, SL.omega, s, SL.r32);
          cudaEventRecord(e0, s);
          for (int w = 0; w < 5 && rc == RAV_OK; ++w) rc = apply_with_omega(sm, l, L.r, L.x, SL.omega, s, SL.r32);
          cudaEventRecord(e1, s);
          float ts = 0.f;
          if (rc == RAV_OK &&
              (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ts, e0, e1) != cudaSuccess))
            rc = RAV_ERR_CUDA;
          if (rc == RAV_OK && ts < tb) {
            tb = ts;
            sbest = splits[ci];
            cbest = tc;
          }
        }
      if (rc == RAV_OK) rc = staged_build(sm, l, sbest, s, cbest);
    }
    cudaMemsetAsync(L.x, 0, sizeof(double) * L.g.n, s);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// Used by the fused smoothing step, which reads the grouping of one thread per owned node.
int regroup_split1(rav_smoother* sm, int level, cudaStream_t s) {
  if (!sm->lev[level].factored) return RAV_OK;
  return regroup(sm, level, 1, s);
}

extern "C" int rav_set_apply_split(rav_smoother* sm, int level, int split, rav_stream stream) {
  if (!sm || level < 1 || level >= sm->mg->nlev) return RAV_ERR_ARG;
  SmLevel& SL = sm->lev[level];
  if (sm->mg->elem == RAV_ELEM_Q1Q1) return split == 1 ? RAV_OK : RAV_ERR_ARG;  // one thread per subdomain
  const int NON = sm->mg->dim == 2 ? 4 : 8;
  if (!SL.factored || split < 1 || split > 32 / NON || (split & (split - 1))) return RAV_ERR_ARG;
  if (split == SL.split) return RAV_OK;
  cudaStream_t s = S(stream);
  RAV_CUDA(cudaStreamSynchronize(s));
  drop_graphs(sm->mg, sm);  // captured cycles hold the old launch shape
  return regroup(sm, level, split, s);
}

extern "C" int rav_set_apply_staged(rav_smoother* sm, int level, int threads_per_subdomain, rav_stream stream) {
  if (!sm || level < 1 || level >= sm->mg->nlev) return RAV_ERR_ARG;
  SmLevel& SL = sm->lev[level];
  const int nt = threads_per_subdomain;
  if (sm->mg->elem != RAV_ELEM_Q2Q1 || !SL.factored || sm->prec == RAV_F64) return nt == 0 ? RAV_OK : RAV_ERR_ARG;
  const bool ok = nt == 0 || nt == 1 || nt == 2 || (sm->mg->dim == 3 && nt == 4);
  if (!ok) return RAV_ERR_ARG;
  if (nt == SL.staged) return RAV_OK;
  cudaStream_t s = S(stream);
  RAV_CUDA(cudaStreamSynchronize(s));
  drop_graphs(sm->mg, sm);  // captured cycles hold the old kernel
  RAV_TRY(staged_build(sm, level, nt, s));
  RAV_CUDA(cudaStreamSynchronize(s));
  return RAV_OK;
}

extern "C" int rav_get_apply_staged(const rav_smoother* sm, int level) {
  if (!sm || level < 1 || level >= sm->mg->nlev) return RAV_ERR_ARG;
  return sm->lev[level].staged;
}

extern "C" int rav_get_apply_split(const rav_smoother* sm, int level) {
  if (!sm || level < 1 || level >= sm->mg->nlev) return RAV_ERR_ARG;
  return sm->lev[level].split;
}

extern "C" int rav_set_patch_omega(rav_smoother* sm, int level, const float* w, rav_stream stream) {
  if (!sm || !w || level < 1 || level >= sm->mg->nlev) return RAV_ERR_ARG;
  const int64_t n = sm->lev[level].np;
  k_f32_to_f64<<<grid_for(n, 256), 256, 0, S(stream)>>>(w, n, sm->lev[level].omega);
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

template <int D, typename T>
static void launch_fact(const SmLevel& SL, const Geo& g, unsigned gb, const double* omega, const void* r, double* x,
                        cudaStream_t s) {
  const T* kinv = (const T*)SL.inv;
  const T* ws = (const T*)SL.ws;
  const AccT<T>* rr = (const AccT<T>*)r;
  switch (SL.split) {
    case 1: k_rav_apply_fact<D, T, 1><<<gb, 128, 0, s>>>(g, kinv, ws, omega, rr, x, SL.units); break;
    case 2: k_rav_apply_fact<D, T, 2><<<gb, 128, 0, s>>>(g, kinv, ws, omega, rr, x, SL.units); break;
    case 4: k_rav_apply_fact<D, T, 4><<<gb, 128, 0, s>>>(g, kinv, ws, omega, rr, x, SL.units); break;
    default:
      if constexpr (D == 2) k_rav_apply_fact<D, T, 8><<<gb, 128, 0, s>>>(g, kinv, ws, omega, rr, x, SL.units);
      break;
  }
}

int apply_with_omega(rav_smoother* sm, int level, const double* r, double* x, const double* omega, cudaStream_t s,
                     const float* r32) {
  rav_mg* mg = sm->mg;
  Level& L = mg->lev[level];
  SmLevel& SL = sm->lev[level];
  const Geo& g = L.g;
  const int D = g.dim;
  if (SL.r32 && !r32) {
    k_f64_to_f32<<<grid_for(g.n, 256), 256, 0, s>>>(r, g.n, SL.r32);
    note_launch();
    r32 = SL.r32;
  }
  cudaEvent_t e0 = nullptr;
  RAV_TRY(prof_begin(mg, level, PROF_APPLY, s, &e0));
  if (g.q == 1 && sm->kind == RAV_AV) {
    const unsigned gb = (unsigned)((g.n_p + 3) / 4);
    const int gg = (int)((g.n + 255) / 256);
    if (D == 2) {
      k_av_q1_corr<2><<<gb, 128, 0, s>>>(g, (double*)SL.inv, omega, r, SL.corr);
      k_av_q1_gather<2><<<gg, 256, 0, s>>>(g, SL.corr, x);
    } else {
      k_av_q1_corr<3><<<gb, 128, 0, s>>>(g, (double*)SL.inv, omega, r, SL.corr);
      k_av_q1_gather<3><<<gg, 256, 0, s>>>(g, SL.corr, x);
    }
    note_launch(2);
  } else if (g.q == 1 && !SL.factored) {
    const unsigned gb = (unsigned)((SL.np + 127) / 128);
    const void* rr = sm->prec == RAV_F64_ROWS ? (const void*)r : (const void*)r32;
#define RAV_APPLY_Q1R(DD, T)                                                                              \
  k_rav_apply_q1_rows<DD, T><<<gb, 128, 0, s>>>(g, (const T*)SL.inv, SL.scale, omega, (const AccT<T>*)rr, x, \
                                                SL.np)
#define RAV_APPLY_Q1R_D(DD)                                  \
  switch (sm->prec) {                                        \
    case RAV_F64_ROWS: RAV_APPLY_Q1R(DD, double); break;     \
    case RAV_F32: RAV_APPLY_Q1R(DD, float); break;           \
    case RAV_BF16: RAV_APPLY_Q1R(DD, __nv_bfloat16); break;  \
    default: RAV_APPLY_Q1R(DD, fp8_t); break;                \
  }
    if (D == 2) {
      RAV_APPLY_Q1R_D(2)
    } else {
      RAV_APPLY_Q1R_D(3)
    }
#undef RAV_APPLY_Q1R_D
#undef RAV_APPLY_Q1R
    note_launch();
  } else if (g.q == 1) {
    const unsigned gb = (unsigned)((SL.np + 127) / 128);
#define RAV_APPLY_Q1(DD, T) \
  k_rav_apply_q1<DD, T><<<gb, 128, 0, s>>>(g, (const T*)SL.inv, omega, (const AccT<T>*)rr, x, SL.np)
    const void* rr = sm->prec == RAV_F64 ? (const void*)r : (const void*)r32;
    if (D == 2) {
      if (sm->prec == RAV_F64) RAV_APPLY_Q1(2, double);
      else if (sm->prec == RAV_F32_FACT) RAV_APPLY_Q1(2, float);
      else RAV_APPLY_Q1(2, __nv_bfloat16);
    } else {
      if (sm->prec == RAV_F64) RAV_APPLY_Q1(3, double);
      else if (sm->prec == RAV_F32_FACT) RAV_APPLY_Q1(3, float);
      else RAV_APPLY_Q1(3, __nv_bfloat16);
    }
#undef RAV_APPLY_Q1
    note_launch();
  } else if (sm->kind == RAV_AV) {
    const unsigned gb = (unsigned)((g.n_p + 3) / 4);
    const int gg = (int)((g.n + 255) / 256);
    if (D == 2) {
      k_av_corr<2><<<gb, 128, 0, s>>>(g, (double*)SL.inv, omega, r, SL.corr);
      k_av_gather<2><<<gg, 256, 0, s>>>(g, SL.corr, x);
    } else {
      k_av_corr<3><<<gb, 128, 0, s>>>(g, (double*)SL.inv, omega, r, SL.corr);
      k_av_gather<3><<<gg, 256, 0, s>>>(g, SL.corr, x);
    }
    note_launch(2);
  } else if (SL.factored && SL.staged) {
    staged_launch(sm, level, omega, r32, x, s);
    note_launch();
  } else if (SL.factored) {
    const unsigned gbs = (unsigned)((SL.units * SL.split + 127) / 128);
    const void* rr = sm->prec == RAV_F64 ? (const void*)r : (const void*)r32;
    if (D == 2) {
      if (sm->prec == RAV_F64) launch_fact<2, double>(SL, g, gbs, omega, rr, x, s);
      else if (sm->prec == RAV_F32_FACT) launch_fact<2, float>(SL, g, gbs, omega, rr, x, s);
      else launch_fact<2, __nv_bfloat16>(SL, g, gbs, omega, rr, x, s);
    } else {
      if (sm->prec == RAV_F64) launch_fact<3, double>(SL, g, gbs, omega, rr, x, s);
      else if (sm->prec == RAV_F32_FACT) launch_fact<3, float>(SL, g, gbs, omega, rr, x, s);
      else launch_fact<3, __nv_bfloat16>(SL, g, gbs, omega, rr, x, s);
    }
    note_launch();
  } else {
    const unsigned gb = (unsigned)((SL.units + 127) / 128);
#define RAV_APPLY(DD, T)                                                                                    \
  k_rav_apply<DD, T><<<gb, 128, 0, s>>>(g, (const T*)SL.inv, SL.scale, omega,                               \
                                        (const AccT<T>*)(std::is_same<T, double>::value ? (const void*)r    \
                                                                                        : (const void*)r32), \
                                        x, SL.units)
    if (D == 2) {
      switch (sm->prec) {
        case RAV_F64_ROWS: RAV_APPLY(2, double); break;
        case RAV_F32: RAV_APPLY(2, float); break;
        case RAV_BF16: RAV_APPLY(2, __nv_bfloat16); break;
        default: RAV_APPLY(2, fp8_t); break;
      }
    } else {
      switch (sm->prec) {
        case RAV_F64_ROWS: RAV_APPLY(3, double); break;
        case RAV_F32: RAV_APPLY(3, float); break;
        case RAV_BF16: RAV_APPLY(3, __nv_bfloat16); break;
        default: RAV_APPLY(3, fp8_t); break;
      }
    }
#undef RAV_APPLY
    note_launch();
  }
  RAV_CUDA(cudaGetLastError());
  RAV_TRY(prof_end(mg, level, PROF_APPLY, e0, s));
  return RAV_OK;
}

static int apply_impl(rav_smoother* sm, int level, const double* r, double* x, cudaStream_t s,
                      const float* r32 = nullptr) {
  if (sm->collect) RAV_TRY(collect_labels(sm, level, r, s));
  return apply_with_omega(sm, level, r, x, sm->lev[level].omega, s, r32);
}

int reset_omega(rav_smoother* sm, cudaStream_t s) {
  for (int l = 1; l < sm->mg->nlev; ++l) {
    k_fill<<<grid_for(sm->lev[l].np, 256), 256, 0, s>>>(sm->lev[l].omega, sm->lev[l].np, sm->omega);
    RAV_CUDA(cudaGetLastError());
  }
  return RAV_OK;
}

int rav_smooth_impl(rav_smoother* sm, int level, double* x, const double* b, int steps, cudaStream_t s,
                    int entry) {
  rav_mg* mg = sm->mg;
  Level& L = mg->lev[level];
  SmLevel& SL = sm->lev[level];
  const Geo& g = L.g;
  const int D = g.dim;
  if (sm->fused && !sm->collect) return fused_smooth_impl(sm, level, x, b, steps, s);
  for (int it = 0; it < steps; ++it) {
    if (sm->kind == RAV_MV_COLOURED) {
      const int ncol = D == 2 ? 16 : 64;
      cudaEvent_t e0;
      RAV_TRY(prof_begin(mg, level, PROF_APPLY, s, &e0));
      for (int c = 0; c < ncol; ++c) {
        int cnt = 1;
        for (int d = 0; d < D; ++d) {
          const int cd = (c >> (2 * d)) & 3;
          cnt *= cd <= g.N ? (g.N - cd) / 4 + 1 : 0;
        }
        if (cnt == 0) continue;
        const unsigned gb = (unsigned)((cnt + 3) / 4);
        if (g.q == 1) {
          if (D == 2) k_mv_q1_colour<2><<<gb, 128, 0, s>>>(g, L.rp, L.ci, L.va, (double*)SL.inv, SL.omega, b, x, c);
          else k_mv_q1_colour<3><<<gb, 128, 0, s>>>(g, L.rp, L.ci, L.va, (double*)SL.inv, SL.omega, b, x, c);
        } else if (D == 2) {
          k_mv_colour<2><<<gb, 128, 0, s>>>(g, L.rp, L.ci, L.va, (double*)SL.inv, SL.omega, b, x, c);
        } else {
          k_mv_colour<3><<<gb, 128, 0, s>>>(g, L.rp, L.ci, L.va, (double*)SL.inv, SL.omega, b, x, c);
        }
        note_launch();
      }
      RAV_CUDA(cudaGetLastError());
      RAV_TRY(prof_end(mg, level, PROF_APPLY, e0, s));
      continue;
    }
    if (it == 0 && entry == ENTRY_X_ZERO) {
      // r = b - L 0 = b on free rows; b is 0 on Dirichlet rows of a coarse level
      RAV_TRY(apply_impl(sm, level, b, x, s));
      continue;
    }
    if (it == 0 && entry == ENTRY_R_READY) {  // r = b - L x is already in L.r (and r32)
      RAV_TRY(apply_impl(sm, level, L.r, x, s, SL.r32));
      continue;
    }
    RAV_TRY(residual_impl(mg, level, x, b, L.r, nullptr, s, SL.r32));
    RAV_TRY(apply_impl(sm, level, L.r, x, s, SL.r32));
    RAV_CUDA(cudaGetLastError());
  }
  return RAV_OK;
}

extern "C" int vanka_apply(rav_smoother* sm, int level, const double* r, double* x, rav_stream stream) {
  if (!sm || !x || !r || level < 1 || level >= sm->mg->nlev || sm->kind == RAV_MV_COLOURED) return RAV_ERR_ARG;
  return apply_impl(sm, level, r, x, S(stream));
}

extern "C" int vanka_smooth(rav_smoother* sm, int level, double* x, const double* b, int steps, rav_stream stream) {
  if (!sm || !x || !b || level < 1 || level >= sm->mg->nlev || steps < 0) return RAV_ERR_ARG;
  return rav_smooth_impl(sm, level, x, b, steps, S(stream));
}

extern "C" int rav_get_patch_counts(const rav_smoother* sm, int level, int64_t out[2]) {
  if (!sm || !out || level < 1 || level >= sm->mg->nlev) return RAV_ERR_ARG;
  const Geo& g = sm->mg->lev[level].g;
  // closed form: per axis the box positions inside the domain interior
  // (Q2-Q1: nodes 2v-2 .. 2v+2; Q1-Q1: vertices v-1 .. v+1)
  int64_t tot = 0;
  std::vector<int64_t> per(g.N + 1);
  const int nb = g.q == 1 ? 3 : 5;
  for (int v = 0; v <= g.N; ++v) {
    int c = 0;
    for (int a = 0; a < nb; ++a) {
      const int J = g.q * v - g.q + a;
      c += (J >= 1 && J <= (int)g.M - 2);
    }
    per[v] = c;
  }
  if (g.dim == 2) {
    for (int v1 = 0; v1 <= g.N; ++v1)
      for (int v0 = 0; v0 <= g.N; ++v0) tot += 2 * per[v0] * per[v1] + 1;
  } else {
    for (int v2 = 0; v2 <= g.N; ++v2)
      for (int v1 = 0; v1 <= g.N; ++v1)
        for (int v0 = 0; v0 <= g.N; ++v0) tot += 3 * per[v0] * per[v1] * per[v2] + 1;
  }
  out[0] = g.n_p;
  out[1] = tot;
  return RAV_OK;
}

extern "C" int rav_get_patches(const rav_smoother* sm, int level, int32_t* off, int32_t* dofs, int32_t* owner,
                               rav_stream stream) {
  if (!sm || level < 1 || level >= sm->mg->nlev || !off || !dofs || !owner) return RAV_ERR_ARG;
  const Geo& g = sm->mg->lev[level].g;
  cudaStream_t s = S(stream);
  int32_t* cnt = nullptr;
  RAV_CUDA(cudaMallocAsync(&cnt, sizeof(int32_t) * g.n_p, s));
  const int gb = (int)((g.n_p + 127) / 128);
  if (g.q == 1) {
    if (g.dim == 2) k_q1_patch_count<2><<<gb, 128, 0, s>>>(g, cnt);
    else k_q1_patch_count<3><<<gb, 128, 0, s>>>(g, cnt);
  } else {
    if (g.dim == 2) k_patch_count<2><<<gb, 128, 0, s>>>(g, cnt);
    else k_patch_count<3><<<gb, 128, 0, s>>>(g, cnt);
  }
  k_scan_i32<<<1, 32, 0, s>>>(cnt, g.n_p, off);
  if (g.q == 1) {
    if (g.dim == 2) k_q1_patch_list<2><<<gb, 128, 0, s>>>(g, off, dofs);
    else k_q1_patch_list<3><<<gb, 128, 0, s>>>(g, off, dofs);
  } else {
    if (g.dim == 2) k_patch_list<2><<<gb, 128, 0, s>>>(g, off, dofs);
    else k_patch_list<3><<<gb, 128, 0, s>>>(g, off, dofs);
  }
  k_owner<<<(int)((g.n + 255) / 256), 256, 0, s>>>(g, owner);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(cnt, s);
  RAV_CUDA(e);
  return RAV_OK;
}

extern "C" int rav_get_inverse_rows(const rav_smoother* sm, int level, int64_t first, int64_t count, double* out,
                                    rav_stream stream) {
  if (!sm || !out || level < 1 || level >= sm->mg->nlev) return RAV_ERR_ARG;
  const SmLevel& SL = sm->lev[level];
  const Geo& g = sm->mg->lev[level].g;
  if (first < 0 || count < 0 || first + count > SL.np) return RAV_ERR_ARG;
  if (count == 0) return RAV_OK;
  cudaStream_t s = S(stream);
  const unsigned gb = (unsigned)count;
  if (g.q == 1 && sm->kind != RAV_RAV) {
    if (g.dim == 2) k_export_q1_full<2><<<gb, 256, 0, s>>>(g, (const double*)SL.inv, first, count, out);
    else k_export_q1_full<3><<<gb, 256, 0, s>>>(g, (const double*)SL.inv, first, count, out);
  } else if (g.q == 1 && !SL.factored) {
#define RAV_EXP_Q1R(DD, T) \
  k_export_q1_rows<DD, T><<<gb, 128, 0, s>>>(g, (const T*)SL.inv, SL.scale, SL.np, first, count, out)
#define RAV_EXP_Q1R_D(DD)                                  \
  switch (sm->prec) {                                      \
    case RAV_F64_ROWS: RAV_EXP_Q1R(DD, double); break;     \
    case RAV_F32: RAV_EXP_Q1R(DD, float); break;           \
    case RAV_BF16: RAV_EXP_Q1R(DD, __nv_bfloat16); break;  \
    default: RAV_EXP_Q1R(DD, fp8_t); break;                \
  }
    if (g.dim == 2) {
      RAV_EXP_Q1R_D(2)
    } else {
      RAV_EXP_Q1R_D(3)
    }
#undef RAV_EXP_Q1R_D
#undef RAV_EXP_Q1R
  } else if (g.q == 1) {
#define RAV_EXP_Q1(DD, T) k_export_q1<DD, T><<<gb, 128, 0, s>>>(g, (const T*)SL.inv, SL.np, first, count, out)
    if (sm->prec == RAV_F64) {
      if (g.dim == 2) RAV_EXP_Q1(2, double);
      else RAV_EXP_Q1(3, double);
    } else if (sm->prec == RAV_F32_FACT) {
      if (g.dim == 2) RAV_EXP_Q1(2, float);
      else RAV_EXP_Q1(3, float);
    } else {
      if (g.dim == 2) RAV_EXP_Q1(2, __nv_bfloat16);
      else RAV_EXP_Q1(3, __nv_bfloat16);
    }
#undef RAV_EXP_Q1
  } else if (sm->kind != RAV_RAV) {
    if (g.dim == 2) k_export_full<2><<<gb, 256, 0, s>>>(g, (const double*)SL.inv, first, count, out);
    else k_export_full<3><<<gb, 256, 0, s>>>(g, (const double*)SL.inv, first, count, out);
  } else if (SL.factored) {
#define RAV_EXP_F(DD, T)                                                                              \
  k_export_fact<DD, T><<<gb, 256, 0, s>>>(g, (const T*)SL.inv, (const T*)SL.ws, first, count, out, \
                                          5 - ilog2(SL.split))
    if (sm->prec == RAV_F64) {
      if (g.dim == 2) RAV_EXP_F(2, double);
      else RAV_EXP_F(3, double);
    } else if (sm->prec == RAV_F32_FACT) {
      if (g.dim == 2) RAV_EXP_F(2, float);
      else RAV_EXP_F(3, float);
    } else {
      if (g.dim == 2) RAV_EXP_F(2, __nv_bfloat16);
      else RAV_EXP_F(3, __nv_bfloat16);
    }
#undef RAV_EXP_F
  } else {
#define RAV_EXP(DD, T) k_export_rav<DD, T><<<gb, 256, 0, s>>>(g, (const T*)SL.inv, SL.scale, first, count, out)
    if (g.dim == 2) {
      switch (sm->prec) {
        case RAV_F64_ROWS: RAV_EXP(2, double); break;
        case RAV_F32: RAV_EXP(2, float); break;
        case RAV_BF16: RAV_EXP(2, __nv_bfloat16); break;
        default: RAV_EXP(2, fp8_t); break;
      }
    } else {
      switch (sm->prec) {
        case RAV_F64_ROWS: RAV_EXP(3, double); break;
        case RAV_F32: RAV_EXP(3, float); break;
        case RAV_BF16: RAV_EXP(3, __nv_bfloat16); break;
        default: RAV_EXP(3, fp8_t); break;
      }
    }
#undef RAV_EXP
  }
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

