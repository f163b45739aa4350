// Fused restricted additive Vanka step on the stabilised Q1-Q1 element (fp64
// factored storage): the residual of Eq. 10 and the subdomain corrections of
// Eq. 13 in one kernel per smoothing step.
//
// A block takes a tile of vertices.  It computes r = b - L x on every box
// vertex of its tile's subdomains (the tile plus a halo of one vertex per
// side, whose rows the neighbouring tiles compute as well) and the pressure
// rows of the tile, keeps them in shared memory, and applies the stored
// factored inverses (centre row of K^{-1}, w, 1/s; structure of arrays) to
// them.  x is double-buffered: a step reads x_in and writes every entry of
// x_out (owned DoFs corrected, Dirichlet ones copied), so a tile never sees
// another tile's update within the step, as the additive method requires.
// The residual rows come from the level's sliced-ELL copy (through the
// row -> slot map; consecutive rows of a tile sit in consecutive slots, so a
// warp's loads stay coalesced) and add in the order of the residual kernel;
// per subdomain the corrections add in the order of the apply kernel.
#include "box.cuh"
#include "common.cuh"
#include "fmt.cuh"

namespace rav {

template <int D>
struct FTile;
template <>
struct FTile<2> {
  static constexpr int X = 16, Y = 16, Z = 1;
};
template <>
struct FTile<3> {
  static constexpr int X = 8, Y = 8, Z = 4;
};

template <int D>
__global__ void __launch_bounds__(256) k_fused_q1(Geo g, const int32_t* __restrict__ sslot,
                                                  const int64_t* __restrict__ sptr, const int32_t* __restrict__ slen,
                                                  const int32_t* __restrict__ scol, const double* __restrict__ sval,
                                                  const double* __restrict__ st, const double* __restrict__ omega,
                                                  const double* __restrict__ b, const double* __restrict__ xin,
                                                  double* __restrict__ xout) {
  using T = FTile<D>;
  constexpr int NV = D == 2 ? 9 : 27, NF = NV * (D + 1) + 1, CEN = D == 2 ? 4 : 13;
  constexpr int UX = T::X + 2, UY = T::Y + 2, UZ = D == 3 ? T::Z + 2 : 1;
  constexpr int NU = UX * UY * UZ;        // box vertices of the tile's subdomains
  constexpr int NT = T::X * T::Y * T::Z;  // tile vertices, one thread each
  __shared__ double ru[NU * D];
  __shared__ double rpr[NT];
  const int N = g.N;
  const int64_t N1 = N + 1;
  const int ox = blockIdx.x * T::X, oy = blockIdx.y * T::Y, oz = D == 3 ? blockIdx.z * T::Z : 0;
  const int tid = threadIdx.x;
  // residual rows: velocity of the free box vertices, pressure of the tile's vertices
  for (int e = tid; e < NU * D + NT; e += NT) {
    int64_t row = -1;
    if (e < NU * D) {
      const int u = e / D, c = e % D;
      const int J0 = ox - 1 + u % UX, J1 = oy - 1 + (u / UX) % UY, J2 = D == 3 ? oz - 1 + u / (UX * UY) : 0;
      bool fr = J0 >= 1 && J0 <= N - 1 && J1 >= 1 && J1 <= N - 1;
      if (D == 3) fr = fr && J2 >= 1 && J2 <= N - 1;
      if (fr) row = D * (J0 + N1 * (J1 + N1 * J2)) + c;
    } else {
      const int t = e - NU * D;
      const int v0 = ox + t % T::X, v1 = oy + (t / T::X) % T::Y, v2 = oz + t / (T::X * T::Y);
      if (v0 <= N && v1 <= N && (D == 2 || v2 <= N)) row = g.n_u + (v0 + N1 * (v1 + N1 * v2));
    }
    double val = 0.0;
    if (row >= 0) {
      const int32_t slot = sslot[row];
      const int64_t sl = slot >> 5;
      const int len = slen[sl];
      const int32_t* c = scol + sptr[sl] + (slot & 31);
      const double* v = sval + sptr[sl] + (slot & 31);
      double a0 = 0.0, a1 = 0.0;
      int k = 0;
      for (; k + 8 <= len; k += 8) {
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          a0 += ld_stream(v + 32 * (k + j)) * xin[ld_stream(c + 32 * (k + j))];
          a1 += ld_stream(v + 32 * (k + j + 1)) * xin[ld_stream(c + 32 * (k + j + 1))];
        }
      }
      for (; k < len; ++k) a0 += ld_stream(v + 32 * k) * xin[ld_stream(c + 32 * k)];
      val = b[row] - (a0 + a1);
    }
    if (e < NU * D) ru[e] = val;
    else rpr[e - NU * D] = val;
  }
  __syncthreads();
  const int tx = tid % T::X, ty = (tid / T::X) % T::Y, tz = tid / (T::X * T::Y);
  const int v0 = ox + tx, v1 = oy + ty, v2 = oz + tz;
  if (v0 > N || v1 > N || (D == 3 && v2 > N)) return;
  const int64_t p = v0 + N1 * (v1 + N1 * v2);
  const int64_t np = g.n_p;
  double y[D], wc[D], t = 0.0;
#pragma unroll
  for (int c = 0; c < D; ++c) y[c] = wc[c] = 0.0;
#pragma unroll
  for (int a2 = 0; a2 < (D == 3 ? 3 : 1); ++a2)
#pragma unroll
    for (int a1 = 0; a1 < 3; ++a1)
#pragma unroll
      for (int a0 = 0; a0 < 3; ++a0) {
        const int n = a0 + 3 * a1 + 9 * a2;
        const int u = (tx + a0) + UX * ((ty + a1) + UY * (tz + a2));
        const double kq = ld_stream(st + n * np + p);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const double wv = ld_stream(st + (NV + n * D + c) * np + p);
          const double rv = ru[u * D + c];
          y[c] += kq * rv;
          t += wv * rv;
          if (n == CEN) wc[c] = wv;
        }
      }
  const double tau = ld_stream(st + (NF - 1) * np + p) * (t - rpr[tid]);
  const double om = omega[p];
  bool cfree = true;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int vd = d == 0 ? v0 : (d == 1 ? v1 : v2);
    cfree &= vd >= 1 && vd <= N - 1;
  }
#pragma unroll
  for (int c = 0; c < D; ++c)
    xout[D * p + c] = cfree ? xin[D * p + c] + om * (y[c] + wc[c] * tau) : xin[D * p + c];
  xout[g.n_u + p] = xin[g.n_u + p] - om * tau;
}

// ---------------------------------------------------------------------------
// The same fusion on Q2-Q1 (Sec. 3's subdomains of 5^d velocity nodes around a
// vertex, Eq. 13 through the block form of L_i^{-1}, factored storage in fp64,
// fp32 or bf16 with one thread per owned node and the grouped layout of
// k_rav_apply_fact with split 1).  A block takes a tile of QX x QY (x QZ)
// vertices; its subdomains' boxes cover the Q2 nodes 2 v0 - 2 ... 2 (v0 + Q)
// per axis ((2Q + 3)^d nodes, a halo of two nodes on each side whose rows the
// neighbouring tiles compute as well).  The block computes r = b - L x on
// those rows (zero on Dirichlet rows and outside the domain) and on the
// pressure rows of its vertices into shared memory, in the accumulation type
// of the storage (fp64, else rounded once to fp32), with the summation order
// of k_residual_sell; then every owned node of the tile's subdomains applies
// its row of K^{-1} as k_rav_apply_fact<D, T, 1> does.  Each Q2 node
// J = 2 v + delta (delta in {0, 1}^d, J <= 2N) is visited by exactly one unit
// of one tile: a free node takes x_in + omega y, a Dirichlet node x_in.
template <int D>
struct QTile;
template <>
struct QTile<2> {
  static constexpr int X = 16, Y = 16, Z = 1;
};
template <>
struct QTile<3> {
  static constexpr int X = 8, Y = 8, Z = 4;
};

template <int D>
struct QTileGeo {
  static constexpr int SX = 2 * QTile<D>::X + 3, SY = 2 * QTile<D>::Y + 3, SZ = D == 3 ? 2 * QTile<D>::Z + 3 : 1;
  static constexpr int NSN = SX * SY * SZ;                             // staged nodes
  static constexpr int NT = QTile<D>::X * QTile<D>::Y * QTile<D>::Z;  // tile vertices
  static constexpr int ROWS = NSN * D + NT;                           // residual rows in shared memory
};

template <int D, typename T>
__global__ void __launch_bounds__(256) k_fused_q2(Geo g, const int32_t* __restrict__ sslot,
                                                  const int64_t* __restrict__ sptr, const int32_t* __restrict__ slen,
                                                  const int32_t* __restrict__ scol, const double* __restrict__ sval,
                                                  const T* __restrict__ kinv, const T* __restrict__ ws,
                                                  const double* __restrict__ omega, const double* __restrict__ b,
                                                  const double* __restrict__ xin, double* __restrict__ xout) {
  using A = AccT<T>;
  using Q = QTileGeo<D>;
  using B = BoxT<D>;
  constexpr int NV = B::NV, NON = B::NON, NWS = D * NV + 1;
  extern __shared__ __align__(16) uint8_t fsm[];
  A* rs = reinterpret_cast<A*>(fsm);  // staged velocity rows (node-major), then the tile's pressure rows
  const int N = g.N;
  const int64_t N1 = N + 1, M = g.M;
  const int ox = blockIdx.x * QTile<D>::X, oy = blockIdx.y * QTile<D>::Y, oz = D == 3 ? blockIdx.z * QTile<D>::Z : 0;
  const int tid = threadIdx.x;
  for (int e = tid; e < Q::ROWS; e += blockDim.x) {
    int64_t row = -1;
    if (e < Q::NSN * D) {
      const int u = e / D, c = e % D;
      const int64_t J0 = 2 * ox - 2 + u % Q::SX, J1 = 2 * oy - 2 + (u / Q::SX) % Q::SY;
      const int64_t J2 = D == 3 ? 2 * oz - 2 + u / (Q::SX * Q::SY) : 0;
      bool fr = J0 >= 1 && J0 <= M - 2 && J1 >= 1 && J1 <= M - 2;
      if (D == 3) fr = fr && J2 >= 1 && J2 <= M - 2;
      if (fr) row = D * (J0 + M * (J1 + M * J2)) + c;
    } else {
      const int t = e - Q::NSN * D;
      const int v0 = ox + t % QTile<D>::X, v1 = oy + (t / QTile<D>::X) % QTile<D>::Y;
      const int v2 = D == 3 ? oz + t / (QTile<D>::X * QTile<D>::Y) : 0;
      if (v0 <= N && v1 <= N && (D == 2 || v2 <= N)) row = g.n_u + (v0 + N1 * (v1 + N1 * v2));
    }
    double rv = 0.0;
    if (row >= 0) {  // as k_residual_sell: eight gathers in flight, two accumulators
      const int32_t slot = sslot[row];
      const int64_t sl = slot >> 5;
      const int len = slen[sl];
      if (len > 1) {
        const int32_t* c = scol + sptr[sl] + (slot & 31);
        const double* v = sval + sptr[sl] + (slot & 31);
        double acc0 = 0.0, acc1 = 0.0;
        int k = 0;
        for (; k + 8 <= len; k += 8) {
          int ck[8];
          double vk[8], xk[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) ck[j] = ld_stream(c + 32 * (k + j));
#pragma unroll
          for (int j = 0; j < 8; ++j) vk[j] = ld_stream(v + 32 * (k + j));
#pragma unroll
          for (int j = 0; j < 8; ++j) xk[j] = xin[ck[j]];
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            acc0 += vk[j] * xk[j];
            acc1 += vk[j + 1] * xk[j + 1];
          }
        }
        for (; k < len; ++k) acc0 += ld_stream(v + 32 * k) * xin[ld_stream(c + 32 * k)];
        rv = b[row] - (acc0 + acc1);
      }
    }
    rs[e] = (A)rv;
  }
  __syncthreads();
  // units: (tile subdomain l, owned node q), 32 / NON subdomains per warp;
  // every lane of a warp runs each pass (its shuffles need them all)
  for (int base_u = 0; base_u < Q::NT * NON; base_u += blockDim.x) {
    const int uu = base_u + tid;
    const int l = uu / NON, q = uu % NON;
    const int lx = l % QTile<D>::X, ly = (l / QTile<D>::X) % QTile<D>::Y, lz = D == 3 ? l / (QTile<D>::X * QTile<D>::Y) : 0;
    int v[3] = {ox + lx, oy + ly, oz + lz};
    const bool live = uu < Q::NT * NON && v[0] <= N && v[1] <= N && (D == 2 || v[2] <= N);
    const int64_t p = live ? v[0] + N1 * (v[1] + N1 * v[2]) : 0;
    const int64_t u = p * NON + q;
    const T* kp = kinv + ((u >> 5) * NV) * 32 + (u & 31);
    const int sb = ((D == 3 ? 2 * lz * Q::SY : 0) + 2 * ly) * Q::SX + 2 * lx;  // staged node of box corner
    A y[D];
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = 0;
    int n = 0;
    for (int a2 = 0; a2 < (D == 3 ? 5 : 1); ++a2)
      for (int a1 = 0; a1 < 5; ++a1)
#pragma unroll
        for (int a0 = 0; a0 < 5; ++a0) {
          const A kq = live ? (A)Fmt<T>::dec(ld_stream(kp + n * 32), nullptr) : (A)0;
          const int sn = sb + a0 + Q::SX * (a1 + Q::SY * a2);
#pragma unroll
          for (int c = 0; c < D; ++c) y[c] += kq * rs[sn * D + c];
          ++n;
        }
    // partial w^T r_u over the box nodes m = q, q + 2^d, ...
    const T* wp = ws + p * NWS;
    A t = 0;
    for (int m = q; m < NV && live; m += NON) {
      const int a0 = m % 5, a1 = (m / 5) % 5, a2 = D == 3 ? m / 25 : 0;
      const int sn = sb + a0 + Q::SX * (a1 + Q::SY * a2);
#pragma unroll
      for (int c = 0; c < D; ++c) t += (A)Fmt<T>::dec(wp[m * D + c], nullptr) * rs[sn * D + c];
    }
#pragma unroll
    for (int o = NON / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (!live) continue;
    const A tau = (A)Fmt<T>::dec(wp[NWS - 1], nullptr) * (t - rs[Q::NSN * D + l]);
    const double om = omega[p];
    int64_t J[3] = {0, 0, 0};
    bool in = true, fr = true;
    int mq = 0;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) {
      const int dl = (q >> d) & 1;
      J[d] = 2 * v[d] + dl;
      in &= J[d] <= 2 * N;
      fr &= (J[d] >= 1) & (J[d] <= 2 * N - 1);
      mq = mq * 5 + 2 + dl;
    }
    if (in) {
      const int64_t dof = D * node_id_t<D>(g, J);
#pragma unroll
      for (int c = 0; c < D; ++c)
        xout[dof + c] = fr ? xin[dof + c] + om * (double)(y[c] + (A)Fmt<T>::dec(wp[mq * D + c], nullptr) * tau)
                           : xin[dof + c];
    }
    if (q == 0) xout[g.n_u + p] = xin[g.n_u + p] + om * (double)-tau;
  }
}

template <int D, typename T>
static void launch_fused_q2(const Level& L, const SmLevel& SL, const double* omega, const double* b, const double* xin,
                            double* xout, cudaStream_t s) {
  const int N1 = L.g.N + 1;
  const dim3 grid((N1 + QTile<D>::X - 1) / QTile<D>::X, (N1 + QTile<D>::Y - 1) / QTile<D>::Y,
                  D == 3 ? (N1 + QTile<D>::Z - 1) / QTile<D>::Z : 1);
  const size_t smem = sizeof(AccT<T>) * QTileGeo<D>::ROWS;
  k_fused_q2<D, T><<<grid, 256, smem, s>>>(L.g, L.sslot, L.sptr, L.slen, L.scol, L.sval, (const T*)SL.inv,
                                            (const T*)SL.ws, omega, b, xin, xout);
}

template <int D, typename T>
static int fused_q2_attr() {
  RAV_CUDA(cudaFuncSetAttribute(k_fused_q2<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(AccT<T>) * QTileGeo<D>::ROWS)));
  return RAV_OK;
}

}  // namespace rav

using namespace rav;

int fused_smooth_impl(rav_smoother* sm, int level, double* x, const double* b, int steps, cudaStream_t s) {
  rav_mg* mg = sm->mg;
  const Level& L = mg->lev[level];
  SmLevel& SL = sm->lev[level];
  const Geo& g = L.g;
  if (steps <= 0) return RAV_OK;
  if (!SL.xalt || !L.sslot) return RAV_ERR_ARG;
  double* cur = x;
  double* alt = SL.xalt;
  const int N1 = g.N + 1;
  for (int it = 0; it < steps; ++it) {
    cudaEvent_t e0;
    RAV_TRY(prof_begin(mg, level, PROF_APPLY, s, &e0));
    if (g.q == 2) {
      const bool bf = sm->prec == RAV_BF16_FACT, f32 = sm->prec == RAV_F32_FACT;
      if (g.dim == 2) {
        if (bf) launch_fused_q2<2, __nv_bfloat16>(L, SL, SL.omega, b, cur, alt, s);
        else if (f32) launch_fused_q2<2, float>(L, SL, SL.omega, b, cur, alt, s);
        else launch_fused_q2<2, double>(L, SL, SL.omega, b, cur, alt, s);
      } else {
        if (bf) launch_fused_q2<3, __nv_bfloat16>(L, SL, SL.omega, b, cur, alt, s);
        else if (f32) launch_fused_q2<3, float>(L, SL, SL.omega, b, cur, alt, s);
        else launch_fused_q2<3, double>(L, SL, SL.omega, b, cur, alt, s);
      }
    } else if (g.dim == 2) {
      const dim3 grid((N1 + FTile<2>::X - 1) / FTile<2>::X, (N1 + FTile<2>::Y - 1) / FTile<2>::Y, 1);
      k_fused_q1<2><<<grid, 256, 0, s>>>(g, L.sslot, L.sptr, L.slen, L.scol, L.sval, (const double*)SL.inv,
                                          SL.omega, b, cur, alt);
    } else {
      const dim3 grid((N1 + FTile<3>::X - 1) / FTile<3>::X, (N1 + FTile<3>::Y - 1) / FTile<3>::Y,
                      (N1 + FTile<3>::Z - 1) / FTile<3>::Z);
      k_fused_q1<3><<<grid, 256, 0, s>>>(g, L.sslot, L.sptr, L.slen, L.scol, L.sval, (const double*)SL.inv,
                                          SL.omega, b, cur, alt);
    }
    note_launch();
    RAV_CUDA(cudaGetLastError());
    RAV_TRY(prof_end(mg, level, PROF_APPLY, e0, s));
    double* tmp = cur;
    cur = alt;
    alt = tmp;
  }
  if (cur != x) RAV_CUDA(cudaMemcpyAsync(x, cur, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, s));
  return RAV_OK;
}

int regroup_split1(rav_smoother* sm, int level, cudaStream_t s);

extern "C" int rav_set_fused_smoothing(rav_smoother* sm, int enable) {
  if (!sm) return RAV_ERR_ARG;
  rav_mg* mg = sm->mg;
  if (enable) {
    if (sm->kind != RAV_RAV) return RAV_ERR_ARG;
    if (mg->elem == RAV_ELEM_Q1Q1 && sm->prec != RAV_F64) return RAV_ERR_ARG;
    if (mg->elem == RAV_ELEM_Q2Q1 && sm->prec != RAV_F64 && sm->prec != RAV_F32_FACT && sm->prec != RAV_BF16_FACT)
      return RAV_ERR_ARG;
  }
  RAV_CUDA(cudaDeviceSynchronize());
  drop_graphs(mg, sm);  // captured cycles hold the other smoothing form
  if (enable) {
    for (int l = 1; l < mg->nlev; ++l) {
      SmLevel& SL = sm->lev[l];
      if (!SL.xalt) RAV_CUDA(cudaMalloc(&SL.xalt, sizeof(double) * mg->lev[l].g.n));
      if (mg->elem == RAV_ELEM_Q2Q1) RAV_TRY(regroup_split1(sm, l, nullptr));  // the fused kernel reads split-1 groups
    }
    if (mg->elem == RAV_ELEM_Q2Q1) {
      int rc = RAV_OK;
      if (mg->dim == 2) {
        rc = fused_q2_attr<2, double>();
        if (rc == RAV_OK) rc = fused_q2_attr<2, float>();
        if (rc == RAV_OK) rc = fused_q2_attr<2, __nv_bfloat16>();
      } else {
        rc = fused_q2_attr<3, double>();
        if (rc == RAV_OK) rc = fused_q2_attr<3, float>();
        if (rc == RAV_OK) rc = fused_q2_attr<3, __nv_bfloat16>();
      }
      RAV_TRY(rc);
    }
    RAV_CUDA(cudaDeviceSynchronize());
  }
  sm->fused = enable != 0;
  return RAV_OK;
}
