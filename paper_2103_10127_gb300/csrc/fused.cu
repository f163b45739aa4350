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
    if (g.dim == 2) {
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

extern "C" int rav_set_fused_smoothing(rav_smoother* sm, int enable) {
  if (!sm) return RAV_ERR_ARG;
  rav_mg* mg = sm->mg;
  if (enable && (mg->elem != RAV_ELEM_Q1Q1 || sm->kind != RAV_RAV || sm->prec != RAV_F64)) return RAV_ERR_ARG;
  RAV_CUDA(cudaDeviceSynchronize());
  drop_graphs(mg, sm);  // captured cycles hold the other smoothing form
  if (enable) {
    for (int l = 1; l < mg->nlev; ++l) {
      SmLevel& SL = sm->lev[l];
      if (!SL.xalt) RAV_CUDA(cudaMalloc(&SL.xalt, sizeof(double) * mg->lev[l].g.n));
    }
  }
  sm->fused = enable != 0;
  return RAV_OK;
}
