// Residual (Eq. 10), grid transfers, coarse solve, V-cycle (Sec. 2, Fig. 1)
// and the outer iterations (stationary multigrid and FGMRES, Sec. 4).
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace rav {

// ---------------------------------------------------------------------------
// r = b - L x on free rows, 0 on Dirichlet rows (Eq. 10), on the sliced-ELL
// copy of L: one thread per row, every lane of a
// slice runs the same trip count, so each fp64 FMA instruction is fully used
// (on GB300 an fp64 warp instruction occupies the pipe whatever its active
// lanes).  Slices of length 1 hold the Dirichlet identity rows: r = 0.
// V = double: the fp64 residual.  V = float (levels between the coarsest and
// the finest when rav_set_coarse_residual_f32 is on): fp32 operator values and
// an fp32 copy of x, products summed in fp32, r = b - sum formed in fp64.
template <typename V>
__global__ void __launch_bounds__(256) k_residual_sell(int64_t nslots, const int32_t* __restrict__ sperm,
                                                       const int64_t* __restrict__ sptr,
                                                       const int32_t* __restrict__ slen,
                                                       const int32_t* __restrict__ scol,
                                                       const V* __restrict__ sval,
                                                       const V* __restrict__ x, const double* __restrict__ b,
                                                       double* __restrict__ r, double* __restrict__ part,
                                                       float* __restrict__ r32) {
  // one slice per warp, one slot per thread (no grid-stride loop: the hardware
  // balances the slices of different lengths across the SMs)
  double acc2 = 0.0;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < nslots) {
    const int64_t s = t >> 5;
    const int32_t row = sperm[t];
    const int len = slen[s];
    const int64_t base = sptr[s] + (t & 31);
    V acc0 = 0, acc1 = 0;
    if (len > 1) {
      const int32_t* c = scol + base;
      const V* v = sval + base;
      int k = 0;
      // eight independent gathers in flight per thread, two accumulators
      for (; k + 8 <= len; k += 8) {
        int ck[8];
        V vk[8], xk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) ck[j] = ld_stream(c + 32 * (k + j));
#pragma unroll
        for (int j = 0; j < 8; ++j) vk[j] = ld_stream(v + 32 * (k + j));
#pragma unroll
        for (int j = 0; j < 8; ++j) xk[j] = x[ck[j]];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          acc0 += vk[j] * xk[j];
          acc1 += vk[j + 1] * xk[j + 1];
        }
      }
      for (; k < len; ++k) acc0 += ld_stream(v + 32 * k) * x[ld_stream(c + 32 * k)];
    }
    if (row >= 0) {
      const double rv = len > 1 ? b[row] - (double)(acc0 + acc1) : 0.0;
      r[row] = rv;
      if (r32) r32[row] = (float)rv;  // round to nearest even, for fp32-accumulating applies
      acc2 = rv * rv;
    }
  }
  if (part) {
    const double bs = block_sum(acc2);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
  }
}

// The same with K threads per row, for levels too small to fill the GPU with
// one thread per row: K consecutive warps take one slice, a warp takes 32/K of
// its rows, lane j of a row sums the slots j, j+K, ... and the K partial sums
// meet by shuffles.  A warp touches K rows of the slice's storage, 32/K
// consecutive values in each, so every 32-byte sector it loads is used.
template <int K, typename V>
__global__ void __launch_bounds__(256) k_residual_sell_split(int64_t nslots, const int32_t* __restrict__ sperm,
                                                             const int64_t* __restrict__ sptr,
                                                             const int32_t* __restrict__ slen,
                                                             const int32_t* __restrict__ scol,
                                                             const V* __restrict__ sval,
                                                             const V* __restrict__ x,
                                                             const double* __restrict__ b, double* __restrict__ r,
                                                             double* __restrict__ part, float* __restrict__ r32) {
  double acc2 = 0.0;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gt < nslots * K) {  // nslots * K is a multiple of 32: whole warps in or out
    const int64_t w = gt >> 5;
    const int lane = (int)(gt & 31);
    const int64_t s = w / K;
    const int t = (int)(w % K) * (32 / K) + lane / K;  // row within the slice
    const int j = lane % K;
    const int len = slen[s];
    const int64_t base = sptr[s] + t;
    V acc0 = 0, acc1 = 0;
    if (len > 1) {
      int k = j;
      for (; k + 3 * K < len; k += 4 * K) {
        int ck[4];
        V vk[4], xk[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) ck[i] = ld_stream(scol + base + 32 * (k + i * K));
#pragma unroll
        for (int i = 0; i < 4; ++i) vk[i] = ld_stream(sval + base + 32 * (k + i * K));
#pragma unroll
        for (int i = 0; i < 4; ++i) xk[i] = x[ck[i]];
        acc0 += vk[0] * xk[0];
        acc1 += vk[1] * xk[1];
        acc0 += vk[2] * xk[2];
        acc1 += vk[3] * xk[3];
      }
      for (; k < len; k += K) acc0 += ld_stream(sval + base + 32 * k) * x[ld_stream(scol + base + 32 * k)];
    }
    V acc = acc0 + acc1;
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const int32_t row = sperm[s * 32 + t];
    if (j == 0 && row >= 0) {
      const double rv = len > 1 ? b[row] - (double)acc : 0.0;
      r[row] = rv;
      if (r32) r32[row] = (float)rv;
      acc2 = rv * rv;
    }
  }
  if (part) {
    const double bs = block_sum(acc2);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
  }
}

__global__ void k_sum_parts(const double* __restrict__ part, int np, double* __restrict__ out, int take_sqrt) {
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) v += part[i];
  v = block_sum(v);
  if (threadIdx.x == 0) *out = take_sqrt ? sqrt(v) : v;
}

__global__ void k_dot_parts(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                            double* __restrict__ part) {
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v += a[i] * b[i];
  v = block_sum(v);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// ---------------------------------------------------------------------------
// Transfers with the per-axis tables (see common.cuh, XferTab): a tensor
// product of per-axis lists of nonzero weights, 32-bit indices.
// W = double: fp64; W = float (rav_set_transfers_f32): fp32 weights and coarse
// values, sums in fp32, added to xf in fp64.
template <int D, typename W>
__global__ void k_prolong(Geo gf, Geo gc, XferTabT<W> T, const W* __restrict__ xc, double* __restrict__ xf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int Mf = (int)gf.M, Mc = (int)gc.M, nnf = (int)gf.nnode;
  if (t < nnf) {
    int I[3] = {0, 0, 0}, id = t;
    bool bnd = false;
    for (int a = 0; a < D; ++a) {
      I[a] = id % Mf;
      id /= Mf;
      bnd |= (I[a] == 0) | (I[a] == Mf - 1);
    }
    if (bnd) return;
    const int c0 = T.pc2[0][I[0]], c1 = T.pc2[1][I[1]], c2 = D == 3 ? T.pc2[2][I[2]] : 1;
    // axis-0 entries are the same for every row: loaded once
    int k0[3];
    W w0[3];
#pragma unroll
    for (int j0 = 0; j0 < 3; ++j0) {
      k0[j0] = j0 < c0 ? D * T.pk2[0][3 * I[0] + j0] : 0;
      w0[j0] = j0 < c0 ? T.pw2[0][3 * I[0] + j0] : W(0);
    }
    W acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0;
    for (int j2 = 0; j2 < c2; ++j2) {
      const int K2 = D == 3 ? T.pk2[2][3 * I[2] + j2] : 0;
      const W w2 = D == 3 ? T.pw2[2][3 * I[2] + j2] : W(1);
      for (int j1 = 0; j1 < c1; ++j1) {
        const int K1 = T.pk2[1][3 * I[1] + j1];
        const W w12 = D == 3 ? w2 * T.pw2[1][3 * I[1] + j1] : T.pw2[1][3 * I[1] + j1];
        const int rowbase = D * Mc * (K1 + Mc * K2);
#pragma unroll
        for (int j0 = 0; j0 < 3; ++j0) {
          if (j0 < c0) {
            const W ww = w12 * w0[j0];
            const int base = rowbase + k0[j0];
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] += ww * xc[base + c];
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < D; ++c) xf[(int64_t)D * t + c] += (double)acc[c];
  } else if (t < nnf + (int)gf.n_p) {
    const int Nf1 = gf.N + 1, Nc1 = gc.N + 1;
    int v[3] = {0, 0, 0}, id = t - nnf;
    for (int a = 0; a < D; ++a) { v[a] = id % Nf1; id /= Nf1; }
    const int c0 = T.pc1[0][v[0]], c1 = T.pc1[1][v[1]], c2 = D == 3 ? T.pc1[2][v[2]] : 1;
    W acc = 0;
    for (int j2 = 0; j2 < c2; ++j2) {
      const int K2 = D == 3 ? T.pk1[2][2 * v[2] + j2] : 0;
      const W w2 = D == 3 ? T.pw1[2][2 * v[2] + j2] : W(1);
      for (int j1 = 0; j1 < c1; ++j1) {
        const int K1 = T.pk1[1][2 * v[1] + j1];
        const W w12 = D == 3 ? w2 * T.pw1[1][2 * v[1] + j1] : T.pw1[1][2 * v[1] + j1];
#pragma unroll
        for (int j0 = 0; j0 < 2; ++j0)
          if (j0 < c0)
            acc += w12 * T.pw1[0][2 * v[0] + j0] * xc[gc.n_u + T.pk1[0][2 * v[0] + j0] + Nc1 * (K1 + Nc1 * K2)];
      }
    }
    xf[gf.n_u + (t - nnf)] += (double)acc;
  }
}

// bc = P^T rf: each coarse DoF gathers the fine DoFs whose interpolation
// uses it (fine boundary nodes are not in the lists); 0 on coarse Dirichlet rows.
// tl (1, 2, 4 or 8) consecutive threads share one coarse DoF: thread `sub`
// takes the rows (j2, j1) numbered sub, sub + tl, ... in row-major order and
// the tl partial sums meet by xor shuffles (tl = 1: one thread, rows in order).
// On small levels a single thread's fp64 chain was the whole kernel's time.
// W = double: fp64; W = float (rav_set_transfers_f32): fp32 weights and fine
// residual, sums in fp32, bc written in fp64.
template <int D, typename W>
__global__ void k_restrict_c(Geo gf, Geo gc, XferTabT<W> T, const W* __restrict__ rf, double* __restrict__ bc,
                             int tl) {
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int t = (int)(gt / tl), sub = (int)(gt % tl);
  const int Mf = (int)gf.M, Mc = (int)gc.M, nnc = (int)gc.nnode;
  W acc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = 0;
  if (t < nnc) {
    int K[3] = {0, 0, 0}, id = t;
    bool bnd = false;
    for (int a = 0; a < D; ++a) {
      K[a] = id % Mc;
      id /= Mc;
      bnd |= (K[a] == 0) | (K[a] == Mc - 1);
    }
    if (!bnd) {
      const int c0 = T.rc2[0][K[0]], c1 = T.rc2[1][K[1]], c2 = D == 3 ? T.rc2[2][K[2]] : 1;
      // axis-0 entries are the same for every row: loaded once
      int k0[7];
      W w0[7];
#pragma unroll
      for (int j0 = 0; j0 < 7; ++j0) {
        k0[j0] = j0 < c0 ? D * T.rk2[0][7 * K[0] + j0] : 0;
        w0[j0] = j0 < c0 ? T.rw2[0][7 * K[0] + j0] : W(0);
      }
      for (int pr = sub; pr < c2 * c1; pr += tl) {
        const int j2 = pr / c1, j1 = pr % c1;
        const int I2 = D == 3 ? T.rk2[2][7 * K[2] + j2] : 0;
        const W w2 = D == 3 ? T.rw2[2][7 * K[2] + j2] : W(1);
        const int I1 = T.rk2[1][7 * K[1] + j1];
        const W w12 = D == 3 ? w2 * T.rw2[1][7 * K[1] + j1] : T.rw2[1][7 * K[1] + j1];
        const int64_t rowbase = (int64_t)D * Mf * (I1 + (int64_t)Mf * I2);
        // fixed trip count with a guard: the loads of a row are issued together
#pragma unroll
        for (int j0 = 0; j0 < 7; ++j0) {
          if (j0 < c0) {
            const W ww = w12 * w0[j0];
            const int64_t base = rowbase + k0[j0];
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] += ww * rf[base + c];
          }
        }
      }
    }
  } else if (t < nnc + (int)gc.n_p) {
    const int Nf1 = gf.N + 1, Nc1 = gc.N + 1;
    int K[3] = {0, 0, 0}, id = t - nnc;
    for (int a = 0; a < D; ++a) { K[a] = id % Nc1; id /= Nc1; }
    const int c0 = T.rc1[0][K[0]], c1 = T.rc1[1][K[1]], c2 = D == 3 ? T.rc1[2][K[2]] : 1;
    for (int pr = sub; pr < c2 * c1; pr += tl) {
      const int j2 = pr / c1, j1 = pr % c1;
      const int V2 = D == 3 ? T.rk1[2][3 * K[2] + j2] : 0;
      const W w2 = D == 3 ? T.rw1[2][3 * K[2] + j2] : W(1);
      const int V1 = T.rk1[1][3 * K[1] + j1];
      const W w12 = D == 3 ? w2 * T.rw1[1][3 * K[1] + j1] : T.rw1[1][3 * K[1] + j1];
#pragma unroll
      for (int j0 = 0; j0 < 3; ++j0)
        if (j0 < c0)
          acc[0] += w12 * T.rw1[0][3 * K[0] + j0] * rf[gf.n_u + T.rk1[0][3 * K[0] + j0] + Nf1 * (V1 + (int64_t)Nf1 * V2)];
    }
  }
  // every lane reaches the shuffles (groups of tl lanes are aligned in the warp)
  for (int o = tl >> 1; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o, tl);
  if (sub != 0) return;
  if (t < nnc) {
#pragma unroll
    for (int c = 0; c < D; ++c) bc[(int64_t)D * t + c] = (double)acc[c];
  } else if (t < nnc + (int)gc.n_p) {
    bc[gc.n_u + (t - nnc)] = (double)acc[0];
  }
}

// Q1-Q1 transfers: velocity and pressure share the vertex tables (pc1/pk1/pw1
// and their transposes rc1/rk1/rw1); one thread per vertex carries the d
// velocity components and the pressure.  Prolongation skips fine boundary
// (Dirichlet) velocity nodes; restriction leaves fine boundary velocity nodes
// out of the sums and writes 0 on coarse boundary velocity rows.
template <int D>
__global__ void k_prolong_q1(Geo gf, Geo gc, XferTab T, const double* __restrict__ xc, double* __restrict__ xf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int)gf.n_p) return;
  const int Nf1 = gf.N + 1, Nc1 = gc.N + 1;
  int v[3] = {0, 0, 0}, id = t;
  bool bnd = false;
  for (int a = 0; a < D; ++a) {
    v[a] = id % Nf1;
    id /= Nf1;
    bnd |= (v[a] == 0) | (v[a] == gf.N);
  }
  const int c0 = T.pc1[0][v[0]], c1 = T.pc1[1][v[1]], c2 = D == 3 ? T.pc1[2][v[2]] : 1;
  double acc[D + 1];
#pragma unroll
  for (int c = 0; c <= D; ++c) acc[c] = 0.0;
  for (int j2 = 0; j2 < c2; ++j2) {
    const int K2 = D == 3 ? T.pk1[2][2 * v[2] + j2] : 0;
    const double w2 = D == 3 ? T.pw1[2][2 * v[2] + j2] : 1.0;
    for (int j1 = 0; j1 < c1; ++j1) {
      const int K1 = T.pk1[1][2 * v[1] + j1];
      const double w12 = D == 3 ? w2 * T.pw1[1][2 * v[1] + j1] : T.pw1[1][2 * v[1] + j1];
#pragma unroll
      for (int j0 = 0; j0 < 2; ++j0)
        if (j0 < c0) {
          const double ww = w12 * T.pw1[0][2 * v[0] + j0];
          const int K = T.pk1[0][2 * v[0] + j0] + Nc1 * (K1 + Nc1 * K2);
#pragma unroll
          for (int c = 0; c < D; ++c) acc[c] += ww * xc[(int64_t)D * K + c];
          acc[D] += ww * xc[gc.n_u + K];
        }
    }
  }
  if (!bnd) {
#pragma unroll
    for (int c = 0; c < D; ++c) xf[(int64_t)D * t + c] += acc[c];
  }
  xf[gf.n_u + t] += acc[D];
}

template <int D>
__global__ void k_restrict_q1(Geo gf, Geo gc, XferTab T, const double* __restrict__ rf, double* __restrict__ bc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int)gc.n_p) return;
  const int Nf1 = gf.N + 1, Nc1 = gc.N + 1;
  int K[3] = {0, 0, 0}, id = t;
  bool cbnd = false;
  for (int a = 0; a < D; ++a) {
    K[a] = id % Nc1;
    id /= Nc1;
    cbnd |= (K[a] == 0) | (K[a] == gc.N);
  }
  const int c0 = T.rc1[0][K[0]], c1 = T.rc1[1][K[1]], c2 = D == 3 ? T.rc1[2][K[2]] : 1;
  double acc[D + 1];
#pragma unroll
  for (int c = 0; c <= D; ++c) acc[c] = 0.0;
  for (int j2 = 0; j2 < c2; ++j2) {
    const int V2 = D == 3 ? T.rk1[2][3 * K[2] + j2] : 0;
    const double w2 = D == 3 ? T.rw1[2][3 * K[2] + j2] : 1.0;
    const bool b2 = D == 3 && (V2 == 0 || V2 == gf.N);
    for (int j1 = 0; j1 < c1; ++j1) {
      const int V1 = T.rk1[1][3 * K[1] + j1];
      const double w12 = D == 3 ? w2 * T.rw1[1][3 * K[1] + j1] : T.rw1[1][3 * K[1] + j1];
      const bool b1 = b2 || V1 == 0 || V1 == gf.N;
#pragma unroll
      for (int j0 = 0; j0 < 3; ++j0)
        if (j0 < c0) {
          const int V0 = T.rk1[0][3 * K[0] + j0];
          const double ww = w12 * T.rw1[0][3 * K[0] + j0];
          const int64_t V = V0 + Nf1 * (V1 + (int64_t)Nf1 * V2);
          if (!(b1 || V0 == 0 || V0 == gf.N)) {
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] += ww * rf[(int64_t)D * V + c];
          }
          acc[D] += ww * rf[gf.n_u + V];
        }
    }
  }
#pragma unroll
  for (int c = 0; c < D; ++c) bc[(int64_t)D * t + c] = cbnd ? 0.0 : acc[c];
  bc[gc.n_u + t] = acc[D];
}

// Coarse solve x = C[:, :n] (b masked to free rows): one warp per row.
__global__ void k_mask_free(Geo g, const double* __restrict__ b, double* __restrict__ bm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < g.n) bm[i] = is_dirichlet(g, i) ? 0.0 : b[i];
}
__global__ void k_coarse_gemv(int64_t n, const double* __restrict__ C, const double* __restrict__ bm,
                              double* __restrict__ x, int accumulate) {
  const int64_t m = n + 1;
  const int lane = threadIdx.x & 31;
  const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  double s = 0.0;
  for (int64_t j = lane; j < n; j += 32) s += C[row * m + j] * bm[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = accumulate ? x[row] + s : s;
}

__global__ void k_axpy(int64_t n, double a, const double* __restrict__ xv, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * xv[i];
}
__global__ void k_scale_copy(int64_t n, double a, const double* __restrict__ xv, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * xv[i];
}
// Block partial sums of the nv dot products V_i . w (V: nv vectors of n,
// contiguous): part[i * gridDim.x + block].
__global__ void k_multi_dot_parts(const double* __restrict__ V, const double* __restrict__ w, int64_t n, int nv,
                                  double* __restrict__ part) {
  for (int i = 0; i < nv; ++i) {
    const double* vi = V + (int64_t)i * n;
    double v = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
      v += vi[k] * w[k];
    v = block_sum(v);
    if (threadIdx.x == 0) part[(int64_t)i * gridDim.x + blockIdx.x] = v;
  }
}
// out[i] = sum over np block partials of dot product i (one block per i).
__global__ void k_multi_sum_parts(const double* __restrict__ part, int np, double* __restrict__ out) {
  double v = 0.0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) v += part[(int64_t)blockIdx.x * np + k];
  v = block_sum(v);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}
// w -= sum_i h[i] V_i
__global__ void k_multi_axpy(const double* __restrict__ V, const double* __restrict__ h, int64_t n, int nv,
                             double* __restrict__ w) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[k];
    for (int i = 0; i < nv; ++i) acc -= h[i] * V[(int64_t)i * n + k];
    w[k] = acc;
  }
}


// x rounded to fp32 (to nearest even), the input of the fp32 coarse-level residual.
__global__ void k_x_to_f32(const double* __restrict__ x, int64_t n, float* __restrict__ x32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x32[i] = (float)x[i];
}

// ---------------------------------------------------------------------------
int residual_impl(rav_mg* mg, int level, const double* x, const double* b, double* r, double* norm2_dev,
                  cudaStream_t s, float* r32) {
  const Level& L = mg->lev[level];
  // fp32 operator and x on the levels between the coarsest and the finest
  const bool f32 = mg->coarse_f32 && L.sval32 && level > 0 && level < mg->nlev - 1;
  if (L.rblock && !f32 && ((uintptr_t)x & 15) == 0) {  // node-blocked velocity rows (x read as 16-byte pairs) + pressure rows
    const int64_t blocks = blocked_blocks(L);
    if (norm2_dev && blocks > mg->part_cap) return RAV_ERR_ARG;
    double* part = norm2_dev ? mg->norm_part : nullptr;
    cudaEvent_t e0;
    RAV_TRY(prof_begin(mg, level, PROF_RESIDUAL, s, &e0));
    blocked_launch(L, x, b, r, part, r32, s);
    if (norm2_dev) k_sum_parts<<<1, 256, 0, s>>>(mg->norm_part, (int)blocks, norm2_dev, 1);
    note_launch(norm2_dev ? 3 : 2);
    RAV_CUDA(cudaGetLastError());
    return prof_end(mg, level, PROF_RESIDUAL, e0, s);
  }
  const int64_t nslots = L.nslice * 32;
  const int K = L.rsplit;
  const int blocks = (int)((nslots * K + 255) / 256);
  if (norm2_dev && blocks > mg->part_cap) return RAV_ERR_ARG;
  double* part = norm2_dev ? mg->norm_part : nullptr;
  cudaEvent_t e0;
  RAV_TRY(prof_begin(mg, level, PROF_RESIDUAL, s, &e0));
  if (f32) {
    k_x_to_f32<<<(unsigned)((L.g.n + 255) / 256), 256, 0, s>>>(x, L.g.n, L.x32);
    note_launch();
  }
#define RAV_RES_SPLIT(KK)                                                                                          \
  {                                                                                                                \
    if (f32)                                                                                                       \
      k_residual_sell_split<KK, float><<<blocks, 256, 0, s>>>(nslots, L.sperm, L.sptr, L.slen, L.scol, L.sval32,   \
                                                              L.x32, b, r, part, r32);                             \
    else                                                                                                           \
      k_residual_sell_split<KK, double><<<blocks, 256, 0, s>>>(nslots, L.sperm, L.sptr, L.slen, L.scol, L.sval, x, \
                                                               b, r, part, r32);                                   \
  }
  switch (K) {
    case 2: RAV_RES_SPLIT(2); break;
    case 4: RAV_RES_SPLIT(4); break;
    case 8: RAV_RES_SPLIT(8); break;
    case 16: RAV_RES_SPLIT(16); break;
    case 32: RAV_RES_SPLIT(32); break;
    default:
      if (f32)
        k_residual_sell<float><<<blocks, 256, 0, s>>>(nslots, L.sperm, L.sptr, L.slen, L.scol, L.sval32, L.x32, b, r,
                                                      part, r32);
      else
        k_residual_sell<double><<<blocks, 256, 0, s>>>(nslots, L.sperm, L.sptr, L.slen, L.scol, L.sval, x, b, r,
                                                       part, r32);
  }
#undef RAV_RES_SPLIT
  if (norm2_dev) k_sum_parts<<<1, 256, 0, s>>>(mg->norm_part, blocks, norm2_dev, 1);
  note_launch(norm2_dev ? 2 : 1);
  RAV_CUDA(cudaGetLastError());
  return prof_end(mg, level, PROF_RESIDUAL, e0, s);
}

void launch_residual_rows(int64_t nslots, const int32_t* sperm, const int64_t* sptr, const int32_t* slen,
                          const int32_t* scol, const double* sval, const double* x, const double* b, double* r,
                          double* part, float* r32, cudaStream_t s) {
  k_residual_sell<double><<<(unsigned)((nslots + 255) / 256), 256, 0, s>>>(nslots, sperm, sptr, slen, scol, sval, x, b, r,
                                                                   part, r32);
}

int dot_impl(rav_mg* mg, const double* a, const double* b, int64_t n, double* out_dev, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)mg->part_cap);
  k_dot_parts<<<blocks, 256, 0, s>>>(a, b, n, mg->norm_part);
  k_sum_parts<<<1, 256, 0, s>>>(mg->norm_part, blocks, out_dev, 0);
  note_launch(2);
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

int restrict_impl(rav_mg* mg, int level, const double* rf, double* bc, cudaStream_t s) {
  const Level &F = mg->lev[level], &C = mg->lev[level - 1];
  if (F.g.q == 1) {
    const int blocks = (int)((C.g.n_p + 127) / 128);
    cudaEvent_t e0;
    RAV_TRY(prof_begin(mg, level, PROF_RESTRICT, s, &e0));
    if (F.g.dim == 2) k_restrict_q1<2><<<blocks, 128, 0, s>>>(F.g, C.g, F.tab(), rf, bc);
    else k_restrict_q1<3><<<blocks, 128, 0, s>>>(F.g, C.g, F.tab(), rf, bc);
    note_launch();
    RAV_CUDA(cudaGetLastError());
    return prof_end(mg, level, PROF_RESTRICT, e0, s);
  }
  const int tl = restrict_split(C.g);
  const int64_t tot = (C.g.nnode + C.g.n_p) * tl;
  const int blocks = (int)((tot + 127) / 128);
  cudaEvent_t e0;
  RAV_TRY(prof_begin(mg, level, PROF_RESTRICT, s, &e0));
  if (F.g.dim == 2) k_restrict_c<2, double><<<blocks, 128, 0, s>>>(F.g, C.g, F.tab(), rf, bc, tl);
  else k_restrict_c<3, double><<<blocks, 128, 0, s>>>(F.g, C.g, F.tab(), rf, bc, tl);
  note_launch();
  RAV_CUDA(cudaGetLastError());
  return prof_end(mg, level, PROF_RESTRICT, e0, s);
}

int prolong_impl(rav_mg* mg, int level, const double* xc, double* xf, cudaStream_t s) {
  const Level &F = mg->lev[level], &C = mg->lev[level - 1];
  if (F.g.q == 1) {
    const int blocks = (int)((F.g.n_p + 127) / 128);
    cudaEvent_t e0;
    RAV_TRY(prof_begin(mg, level, PROF_PROLONG, s, &e0));
    if (F.g.dim == 2) k_prolong_q1<2><<<blocks, 128, 0, s>>>(F.g, C.g, F.tab(), xc, xf);
    else k_prolong_q1<3><<<blocks, 128, 0, s>>>(F.g, C.g, F.tab(), xc, xf);
    note_launch();
    RAV_CUDA(cudaGetLastError());
    return prof_end(mg, level, PROF_PROLONG, e0, s);
  }
  const int64_t tot = F.g.nnode + F.g.n_p;
  const int blocks = (int)((tot + 127) / 128);
  cudaEvent_t e0;
  RAV_TRY(prof_begin(mg, level, PROF_PROLONG, s, &e0));
  if (F.g.dim == 2) k_prolong<2, double><<<blocks, 128, 0, s>>>(F.g, C.g, F.tab(), xc, xf);
  else k_prolong<3, double><<<blocks, 128, 0, s>>>(F.g, C.g, F.tab(), xc, xf);
  note_launch();
  RAV_CUDA(cudaGetLastError());
  return prof_end(mg, level, PROF_PROLONG, e0, s);
}

// FP32 transfers of the V-cycle (rav_set_transfers_f32, Q2-Q1): the
// restriction of the fine residual already rounded to fp32 (rf32, written by
// the residual kernel), and the prolongation of the coarse x rounded to fp32
// (one conversion kernel); fp32 weights and sums, fp64 outputs.
static int restrict_f32(rav_mg* mg, int level, const float* rf32, double* bc, cudaStream_t s) {
  const Level &F = mg->lev[level], &C = mg->lev[level - 1];
  const int tl = restrict_split(C.g);
  const int64_t tot = (C.g.nnode + C.g.n_p) * tl;
  const int blocks = (int)((tot + 127) / 128);
  cudaEvent_t e0;
  RAV_TRY(prof_begin(mg, level, PROF_RESTRICT, s, &e0));
  if (F.g.dim == 2) k_restrict_c<2, float><<<blocks, 128, 0, s>>>(F.g, C.g, F.tabs32, rf32, bc, tl);
  else k_restrict_c<3, float><<<blocks, 128, 0, s>>>(F.g, C.g, F.tabs32, rf32, bc, tl);
  note_launch();
  RAV_CUDA(cudaGetLastError());
  return prof_end(mg, level, PROF_RESTRICT, e0, s);
}
static int prolong_f32(rav_mg* mg, int level, const double* xc, double* xf, cudaStream_t s) {
  const Level &F = mg->lev[level], &C = mg->lev[level - 1];
  const int64_t tot = F.g.nnode + F.g.n_p;
  const int blocks = (int)((tot + 127) / 128);
  cudaEvent_t e0;
  RAV_TRY(prof_begin(mg, level, PROF_PROLONG, s, &e0));
  k_x_to_f32<<<(unsigned)((C.g.n + 255) / 256), 256, 0, s>>>(xc, C.g.n, F.xc32);
  if (F.g.dim == 2) k_prolong<2, float><<<blocks, 128, 0, s>>>(F.g, C.g, F.tabs32, F.xc32, xf);
  else k_prolong<3, float><<<blocks, 128, 0, s>>>(F.g, C.g, F.tabs32, F.xc32, xf);
  note_launch(2);
  RAV_CUDA(cudaGetLastError());
  return prof_end(mg, level, PROF_PROLONG, e0, s);
}

// x = C b (overwrite) or x += C b, with b masked to free rows.
static int coarse_apply(rav_mg* mg, const double* b, double* x, int accumulate, cudaStream_t s) {
  Level& L = mg->lev[0];
  const int64_t n = L.g.n;
  double* bm = L.b == b ? L.r : L.b;  // masked copy in whichever work vector is not the input
  if (bm == b) return RAV_ERR_ARG;
  cudaEvent_t e0;
  RAV_TRY(prof_begin(mg, 0, PROF_COARSE, s, &e0));
  k_mask_free<<<(int)((n + 255) / 256), 256, 0, s>>>(L.g, b, bm);
  k_coarse_gemv<<<(int)((n + 7) / 8), 256, 0, s>>>(n, mg->cinv, bm, x, accumulate);
  note_launch(2);
  RAV_CUDA(cudaGetLastError());
  return prof_end(mg, 0, PROF_COARSE, e0, s);
}

int coarse_impl(rav_mg* mg, const double* b, double* x, cudaStream_t s) { return coarse_apply(mg, b, x, 0, s); }

// V(nu1, nu2) on level l with iterate x and right-hand side b.  With
// ENTRY_X_ZERO the first residual below the finest level equals b and the
// coarse correction simply overwrites x; with ENTRY_R_READY the finest
// level's residual vector already holds b - L x.
static int vcycle_rec(rav_mg* mg, rav_smoother* sm, int l, double* x, const double* b, int nu1, int nu2,
                      int entry, cudaStream_t s) {
  Level& L = mg->lev[l];
  if (l == 0) {
    if (entry == ENTRY_X_ZERO) return coarse_apply(mg, b, x, 0, s);
    RAV_TRY(residual_impl(mg, 0, x, b, L.r, nullptr, s));
    return coarse_apply(mg, L.r, x, 1, s);  // x += C r (masked copy of r goes to L.b)
  }
  // below the finest level x enters as 0 and b (a restricted residual) is 0 on
  // Dirichlet rows, so the first smoothing step can take r = b
  const int first = l < mg->nlev - 1 ? (entry == ENTRY_X_ZERO ? ENTRY_X_ZERO : ENTRY_GENERAL)
                                     : (entry == ENTRY_R_READY ? ENTRY_R_READY : ENTRY_GENERAL);
  RAV_TRY(rav_smooth_impl(sm, l, x, b, nu1, s, first));
  Level& C = mg->lev[l - 1];
  const bool xf32 = mg->xfer_f32 && L.rf32;  // fp32 transfers between l and l-1
  RAV_TRY(residual_impl(mg, l, x, b, L.r, nullptr, s, xf32 ? L.rf32 : nullptr));
  RAV_TRY(xf32 ? restrict_f32(mg, l, L.rf32, C.b, s) : restrict_impl(mg, l, L.r, C.b, s));
  RAV_CUDA(cudaMemsetAsync(C.x, 0, sizeof(double) * C.g.n, s));
  RAV_TRY(vcycle_rec(mg, sm, l - 1, C.x, C.b, nu1, nu2, ENTRY_X_ZERO, s));
  RAV_TRY(xf32 ? prolong_f32(mg, l, C.x, x, s) : prolong_impl(mg, l, C.x, x, s));
  RAV_TRY(rav_smooth_impl(sm, l, x, b, nu2, s));
  return RAV_OK;
}

int vcycle_impl(rav_mg* mg, rav_smoother* sm, double* x, const double* b, int nu1, int nu2, int entry,
                cudaStream_t s) {
  return vcycle_rec(mg, sm, mg->nlev - 1, x, b, nu1, nu2, entry, s);
}

// One V-cycle as a CUDA graph.  The first call for a given (smoother, x, b,
// nu1, nu2) captures the cycle's kernels on a private stream; every call
// replays the instantiated graph on the caller's stream, which removes the
// per-kernel launch latency that dominates the small levels.  Not used while
// the timing hook records (its events would be baked into the graph).
static int vcycle_graph(rav_mg* mg, rav_smoother* sm, double* x, const double* b, int nu1, int nu2, int entry,
                        cudaStream_t s) {
  if (!mg->use_graphs || mg->prof_mask != 0 || sm->collect) return vcycle_impl(mg, sm, x, b, nu1, nu2, entry, s);
  rav_mg::GraphEntry* hit = nullptr;
  for (auto& e : mg->graphs)
    if (e.sm == sm && e.x == x && e.b == b && e.nu1 == nu1 && e.nu2 == nu2 && e.entry == entry) hit = &e;
  if (!hit) {
    // capturing runs nothing; the replay on s is ordered after s's earlier work
    if (!mg->cap_stream) RAV_CUDA(cudaStreamCreateWithFlags(&mg->cap_stream, cudaStreamNonBlocking));
    const int64_t l0 = rav_kernel_launches();
    RAV_CUDA(cudaStreamBeginCapture(mg->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = vcycle_impl(mg, sm, x, b, nu1, nu2, entry, mg->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(mg->cap_stream, &graph);
    if (rc != RAV_OK || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (ec != cudaSuccess) note_cuda_error(ec);
      return rc != RAV_OK ? rc : RAV_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    RAV_CUDA(ei);
    if (mg->graphs.size() >= 32) {
      cudaGraphExecDestroy(mg->graphs.front().exec);
      mg->graphs.erase(mg->graphs.begin());
    }
    mg->graphs.push_back({sm, x, b, nu1, nu2, entry, rav_kernel_launches() - l0, exec});
    hit = &mg->graphs.back();
    note_launch((int)-hit->launches);  // counted again below, per replay
  }
  RAV_CUDA(cudaGraphLaunch(hit->exec, s));
  note_launch((int)hit->launches);
  return RAV_OK;
}

void drop_graphs(rav_mg* mg, const rav_smoother* sm) {
  for (size_t i = 0; i < mg->graphs.size();) {
    if (!sm || mg->graphs[i].sm == sm) {
      cudaGraphExecDestroy(mg->graphs[i].exec);
      mg->graphs.erase(mg->graphs.begin() + i);
    } else {
      ++i;
    }
  }
}

static int read_scalar(rav_mg* mg, const double* dev, double* host, cudaStream_t s) {
  RAV_CUDA(cudaMemcpyAsync(mg->scalar_host, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  RAV_CUDA(cudaStreamSynchronize(s));
  *host = mg->scalar_host[0];
  return RAV_OK;
}

}  // namespace rav

using namespace rav;

extern "C" int rav_residual(rav_mg* mg, int level, const double* x, const double* b, double* r, double* norm_host,
                            rav_stream stream) {
  if (!mg || !x || !b || !r || level < 0 || level >= mg->nlev) return RAV_ERR_ARG;
  cudaStream_t s = S(stream);
  RAV_TRY(residual_impl(mg, level, x, b, r, norm_host ? mg->scalar_dev : nullptr, s));
  if (norm_host) RAV_TRY(read_scalar(mg, mg->scalar_dev, norm_host, s));
  return RAV_OK;
}

extern "C" int rav_restrict(rav_mg* mg, int level, const double* rf, double* bc, rav_stream stream) {
  if (!mg || !rf || !bc || level < 1 || level >= mg->nlev) return RAV_ERR_ARG;
  return restrict_impl(mg, level, rf, bc, S(stream));
}

extern "C" int rav_prolong_add(rav_mg* mg, int level, const double* xc, double* xf, rav_stream stream) {
  if (!mg || !xc || !xf || level < 1 || level >= mg->nlev) return RAV_ERR_ARG;
  return prolong_impl(mg, level, xc, xf, S(stream));
}

extern "C" int rav_coarse_solve(rav_mg* mg, const double* b, double* x, rav_stream stream) {
  if (!mg || !b || !x) return RAV_ERR_ARG;
  Level& L = mg->lev[0];
  if (b == L.r || b == L.b) return RAV_ERR_ARG;
  return coarse_impl(mg, b, x, S(stream));
}

extern "C" int vcycle(rav_mg* mg, rav_smoother* sm, double* x, const double* b, int nu1, int nu2,
                      rav_stream stream) {
  if (!mg || !sm || sm->mg != mg || !x || !b || nu1 < 0 || nu2 < 0) return RAV_ERR_ARG;
  return vcycle_graph(mg, sm, x, b, nu1, nu2, ENTRY_GENERAL, S(stream));
}

// ---------------------------------------------------------------------------
// Residual and norm without any allocation, for callers that must not call
// cudaMalloc (code running while a stream is captured into a CUDA graph, or
// real-time loops that work from memory reserved up front).  The per-block
// partial sums of the norm live in this fixed device array instead of the
// hierarchy's work buffer.  Every GPU that loads the library holds the array
// until the process exits.
static constexpr int kNoAllocParts = 16384;  // partial sums: one per 256 rows
static __device__ __align__(256) double g_noalloc_parts[kNoAllocParts];
static constexpr int kMaxDevices = 64;
static double* g_noalloc_addr[kMaxDevices] = {};
static std::mutex g_noalloc_mu;

// Device address of g_noalloc_parts on the current device, which must be the
// device the hierarchy was built on (its pointers are only valid there).  In
// host code the symbol is only a stand-in; the address is looked up once per
// device, with that device current, and remembered.
static int noalloc_parts_address(const rav_mg* mg, double** out) {
  int dev = 0;
  RAV_CUDA(cudaGetDevice(&dev));
  if (dev != mg->device || dev < 0 || dev >= kMaxDevices) return RAV_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    RAV_CUDA(cudaGetSymbolAddress(&p, g_noalloc_parts));
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return RAV_OK;
}

extern "C" int rav_residual_norm_noalloc(rav_mg* mg, int level, const double* x, const double* b, double* r,
                                         double* norm_dev, rav_stream stream) {
  if (!mg || !x || !b || !r || !norm_dev || level < 0 || level >= mg->nlev) return RAV_ERR_ARG;
  const Level& L = mg->lev[level];
  const int64_t nslots = L.nslice * 32;
  const int64_t blocks = (nslots + 255) / 256;
  if (blocks > kNoAllocParts) return RAV_ERR_ARG;  // level has more than 4,194,304 row slots
  double* parts = nullptr;
  RAV_TRY(noalloc_parts_address(mg, &parts));
  cudaStream_t s = S(stream);
  k_residual_sell<double><<<(unsigned)blocks, 256, 0, s>>>(nslots, L.sperm, L.sptr, L.slen, L.scol, L.sval, x, b, r, parts,
                                                   nullptr);
  k_sum_parts<<<1, 256, 0, s>>>(parts, (int)blocks, norm_dev, 1);
  note_launch(2);
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

extern "C" int rav_set_graphs(rav_mg* mg, int enable) {
  if (!mg) return RAV_ERR_ARG;
  mg->use_graphs = enable != 0;
  if (!mg->use_graphs) drop_graphs(mg, nullptr);
  return RAV_OK;
}

// ---------------------------------------------------------------------------
static int solve_stationary(rav_mg* mg, rav_smoother* sm, double* x, const double* b, const rav_solve_opts& o,
                            rav_solve_info* info, cudaStream_t s) {
  Level& L = mg->lev[mg->nlev - 1];
  float* r32 = sm->lev[mg->nlev - 1].r32;
  double r0 = 0.0, rk = 0.0;
  // every norm residual leaves b - L x in L.r (and r32), where the next
  // cycle's first smoothing step takes it instead of recomputing it
  RAV_TRY(residual_impl(mg, mg->nlev - 1, x, b, L.r, mg->scalar_dev, s, r32));
  RAV_TRY(read_scalar(mg, mg->scalar_dev, &r0, s));
  if (info && info->history_host) info->history_host[0] = 1.0;
  if (r0 == 0.0) {
    if (info) { info->iterations = 0; info->final_ratio = 0.0; info->status = RAV_OK; }
    return RAV_OK;
  }
  int rc = RAV_ERR_NOT_CONVERGED, k = 0, fell_back = 0;
  double ratio = 1.0, prev = 1.0;
  for (k = 1; k <= o.maxit; ++k) {
    RAV_TRY(vcycle_graph(mg, sm, x, b, o.nu_pre, o.nu_post, ENTRY_R_READY, s));
    RAV_TRY(residual_impl(mg, mg->nlev - 1, x, b, L.r, mg->scalar_dev, s, r32));
    RAV_TRY(read_scalar(mg, mg->scalar_dev, &rk, s));
    ratio = rk / r0;
    if (info && info->history_host) info->history_host[k] = ratio;
    if (!std::isfinite(ratio)) { rc = RAV_ERR_NAN; break; }
    if (ratio <= o.tol) { rc = RAV_OK; break; }
    if (o.diverge > 0 && ratio > o.diverge) { rc = RAV_ERR_DIVERGED; break; }
    // fallback: a cycle that reduced the residual by less than fallback_rho
    // puts every subdomain back on the fixed damping of vanka_setup
    if (o.fallback_rho > 0 && !fell_back && ratio / prev > o.fallback_rho) {
      RAV_TRY(reset_omega(sm, s));
      fell_back = 1;
    }
    prev = ratio;
  }
  if (info) {
    info->iterations = k > o.maxit ? o.maxit : k;
    info->final_ratio = ratio;
    info->status = rc;
    info->fell_back = fell_back;
  }
  return rc;
}

// FGMRES(m), right-preconditioned by one V-cycle from a zero guess; classical
// Gram-Schmidt applied twice with fused device dot products and updates,
// Givens rotations on the host.  Work vectors: V (m+1 Krylov vectors), Z (m
// preconditioned ones), w, a zero vector, the Hessenberg column and the dot
// products' block partial sums (ndb per vector).
struct FgmresWork {
  double *V = nullptr, *Z = nullptr, *w = nullptr, *zero = nullptr, *hdev = nullptr, *dpart = nullptr;
};
static constexpr int kFgmresDotBlocks = 152 * 2;

static int fgmres_run(rav_mg* mg, rav_smoother* sm, double* x, const double* b, const rav_solve_opts& o,
                      rav_solve_info* info, cudaStream_t s, const FgmresWork& W);

static int solve_fgmres(rav_mg* mg, rav_smoother* sm, double* x, const double* b, const rav_solve_opts& o,
                        rav_solve_info* info, cudaStream_t s) {
  const int64_t n = mg->lev[mg->nlev - 1].g.n;
  const int m = o.restart > 0 ? o.restart : 30;
  FgmresWork W;
  bool ok = cudaMallocAsync(&W.V, sizeof(double) * n * (m + 1), s) == cudaSuccess;
  ok = ok && cudaMallocAsync(&W.Z, sizeof(double) * n * m, s) == cudaSuccess;
  ok = ok && cudaMallocAsync(&W.w, sizeof(double) * n, s) == cudaSuccess;
  ok = ok && cudaMallocAsync(&W.zero, sizeof(double) * n, s) == cudaSuccess;
  ok = ok && cudaMallocAsync(&W.hdev, sizeof(double) * (2 * m + 3), s) == cudaSuccess;
  ok = ok && cudaMallocAsync(&W.dpart, sizeof(double) * kFgmresDotBlocks * (m + 1), s) == cudaSuccess;
  ok = ok && cudaMemsetAsync(W.zero, 0, sizeof(double) * n, s) == cudaSuccess;
  const int rc = ok ? fgmres_run(mg, sm, x, b, o, info, s, W) : RAV_ERR_CUDA;
  for (double* p : {W.V, W.Z, W.w, W.zero, W.hdev, W.dpart})
    if (p) cudaFreeAsync(p, s);
  return rc;
}

static int fgmres_run(rav_mg* mg, rav_smoother* sm, double* x, const double* b, const rav_solve_opts& o,
                      rav_solve_info* info, cudaStream_t s, const FgmresWork& W) {
  const int fine = mg->nlev - 1;
  Level& L = mg->lev[fine];
  const int64_t n = L.g.n;
  const int m = o.restart > 0 ? o.restart : 30;
  double *V = W.V, *Z = W.Z, *w = W.w, *zero = W.zero, *hdev = W.hdev, *dpart = W.dpart;
  const int ndb = kFgmresDotBlocks;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gam(m + 1), y(m);
  const int gb = grid_for(n, 256, 152 * 16);
  double r0 = 0.0, beta = 0.0, ratio = 1.0;
  int it = 0, rc = RAV_ERR_NOT_CONVERGED;
  RAV_TRY(residual_impl(mg, fine, x, b, L.r, mg->scalar_dev, s));
  RAV_TRY(read_scalar(mg, mg->scalar_dev, &r0, s));
  if (info && info->history_host) info->history_host[0] = 1.0;
  if (r0 == 0.0) rc = RAV_OK;
  while (rc == RAV_ERR_NOT_CONVERGED && it < o.maxit) {
    RAV_TRY(residual_impl(mg, fine, x, b, L.r, mg->scalar_dev, s));
    RAV_TRY(read_scalar(mg, mg->scalar_dev, &beta, s));
    if (beta / r0 <= o.tol) { rc = RAV_OK; ratio = beta / r0; break; }
    k_scale_copy<<<gb, 256, 0, s>>>(n, 1.0 / beta, L.r, V);
    note_launch();
    std::fill(gam.begin(), gam.end(), 0.0);
    gam[0] = beta;
    int j = 0;
    bool done = false;
    for (; j < m && it < o.maxit; ++j) {
      double* vj = V + (int64_t)j * n;
      double* zj = Z + (int64_t)j * n;
      // z_j = M v_j: one V-cycle from a zero guess, replayed from a graph on
      // the finest level's own work vectors (fixed pointers: one graph)
      RAV_CUDA(cudaMemcpyAsync(L.b, vj, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      RAV_CUDA(cudaMemsetAsync(L.x, 0, sizeof(double) * n, s));
      RAV_TRY(vcycle_graph(mg, sm, L.x, L.b, o.nu_pre, o.nu_post, ENTRY_X_ZERO, s));
      RAV_CUDA(cudaMemcpyAsync(zj, L.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      // w = L z: the residual of z against a zero right-hand side is -L z
      RAV_TRY(residual_impl(mg, fine, zj, zero, w, nullptr, s));
      k_scale_copy<<<gb, 256, 0, s>>>(n, -1.0, w, w);
      note_launch();
      // classical Gram-Schmidt applied twice (CGS2): h = V^T w, w -= V h, twice,
      // each pass one fused dot kernel and one fused update
      for (int pass = 0; pass < 2; ++pass) {
        double* hp = hdev + pass * (m + 1);
        k_multi_dot_parts<<<ndb, 256, 0, s>>>(V, w, n, j + 1, dpart);
        k_multi_sum_parts<<<j + 1, 256, 0, s>>>(dpart, ndb, hp);
        k_multi_axpy<<<gb, 256, 0, s>>>(V, hp, n, j + 1, w);
        note_launch(3);
      }
      RAV_TRY(dot_impl(mg, w, w, n, hdev + 2 * (m + 1), s));
      RAV_CUDA(cudaMemcpyAsync(mg->scalar_host, hdev, sizeof(double) * (2 * m + 3), cudaMemcpyDeviceToHost, s));
      RAV_CUDA(cudaStreamSynchronize(s));
      for (int i = 0; i <= j; ++i) H[i * m + j] = mg->scalar_host[i] + mg->scalar_host[m + 1 + i];
      const double hn = std::sqrt(mg->scalar_host[2 * (m + 1)]);
      H[(j + 1) * m + j] = hn;
      k_scale_copy<<<gb, 256, 0, s>>>(n, hn > 0 ? 1.0 / hn : 0.0, w, V + (int64_t)(j + 1) * n);
      note_launch();
      for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], bb = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * bb;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      const double a = H[j * m + j], bb = H[(j + 1) * m + j];
      const double den = std::sqrt(a * a + bb * bb);
      cs[j] = a / den;
      sn[j] = bb / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      gam[j + 1] = -sn[j] * gam[j];
      gam[j] = cs[j] * gam[j];
      ++it;
      ratio = std::fabs(gam[j + 1]) / r0;
      if (info && info->history_host) info->history_host[it] = ratio;
      if (!std::isfinite(ratio)) { rc = RAV_ERR_NAN; done = true; ++j; break; }
      if (ratio <= o.tol) { done = true; ++j; break; }
    }
    for (int i = j - 1; i >= 0; --i) {
      double sum = gam[i];
      for (int k = i + 1; k < j; ++k) sum -= H[i * m + k] * y[k];
      y[i] = sum / H[i * m + i];
    }
    for (int i = 0; i < j; ++i) k_axpy<<<gb, 256, 0, s>>>(n, y[i], Z + (int64_t)i * n, x);
    note_launch(j);
    RAV_CUDA(cudaGetLastError());
    if (rc == RAV_ERR_NAN) break;
    if (done) {
      RAV_TRY(residual_impl(mg, fine, x, b, L.r, mg->scalar_dev, s));
      double rt;
      RAV_TRY(read_scalar(mg, mg->scalar_dev, &rt, s));
      ratio = rt / r0;
      if (info && info->history_host) info->history_host[it] = ratio;
      if (ratio <= o.tol) rc = RAV_OK;
    }
  }
  if (info) {
    info->iterations = it;
    info->final_ratio = ratio;
    info->status = rc;
  }
  return rc;
}

extern "C" int solve(rav_mg* mg, rav_smoother* sm, double* x, const double* b, const rav_solve_opts* opts,
                     rav_solve_info* info, rav_stream stream) {
  // info is filled on every exit, failures included: the outer loops set
  // what they reached, and a failure before that leaves these defaults
  if (info) {
    info->iterations = 0;
    info->status = RAV_ERR_ARG;
    info->final_ratio = 1.0;
    info->fell_back = 0;
  }
  int rc = RAV_ERR_ARG;
  if (!mg || !sm || sm->mg != mg || !x || !b || !opts || opts->maxit < 0 || !(opts->tol > 0)) rc = RAV_ERR_ARG;
  else if (opts->outer == 1) rc = opts->restart > 62 ? RAV_ERR_ARG : solve_fgmres(mg, sm, x, b, *opts, info, S(stream));
  else rc = solve_stationary(mg, sm, x, b, *opts, info, S(stream));
  if (info) info->status = rc;
  return rc;
}
