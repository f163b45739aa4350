// Learned per-subdomain damping omega_i (Eq. 11 allows a diagonal weighting
// per subdomain; the paper itself uses one constant).
//
//  * features: 8 numbers per subdomain from the local grid and viscosity;
//  * labels:   omega*_i = clip(omega_i + <r', L c_i> / <L c_i, L c_i>, 0, 1.5),
//              c_i the subdomain's own restricted correction (weight 1),
//              r' = r - L sum_j omega_j c_j the residual after the whole
//              step: the exact minimiser of the post-step residual norm in
//              omega_i alone, averaged over the smoothing steps in which it
//              is collected;
//  * model:    MLP 8 -> 64 -> 64 -> 1 (ReLU, ReLU, 1.5 sigmoid), parameters
//              W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3 (4801);
//              inference with weights rounded to fp16 and fp32 accumulation,
//              training in fp32 (full-batch gradient, Adam).
#include <cuda_fp16.h>

#include <cmath>
#include <vector>

#include "box.cuh"
#include "common.cuh"

namespace rav {

constexpr int kH = 64, kF = 8;
constexpr int kNParam = kH * kF + kH + kH * kH + kH + kH + 1;

// ---------------------------------------------------------------------------
// Features of subdomain p on a level (cells around its vertex):
//  f0 log10(eta_max / eta_min) over their 3^d Gauss points, f1 mean log10 eta,
//  f2 / f3 log10 of the largest / smallest cell aspect ratio (long / short
//  edge), f4 level / (levels - 1), f5 subdomain DoFs / box positions,
//  f6 fraction of in-domain box nodes on the Dirichlet boundary,
//  f7 log10 of the mean cell diagonal.
template <int D>
__global__ void k_features(Geo g, Coef C, int level, int nlev, float* __restrict__ F) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= g.n_p) return;
  int v[3] = {0, 0, 0};
  vertex_of(g, p, v);
  int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) {
    clo[a] = v[a] - 1 < 0 ? 0 : v[a] - 1;
    chi[a] = v[a] > g.N - 1 ? g.N - 1 : v[a];
  }
  const double gx = 0.38729833462074168852;
  double emin = 1e300, emax = 0.0, lsum = 0.0, amax = 0.0, amin = 1e300, diag = 0.0;
  int nq = 0, ncell = 0;
  for (int c2 = (D == 3 ? clo[2] : 0); c2 <= (D == 3 ? chi[2] : 0); ++c2)
    for (int c1 = clo[1]; c1 <= chi[1]; ++c1)
      for (int c0 = clo[0]; c0 <= chi[0]; ++c0) {
        const int c[3] = {c0, c1, c2};
        double lo[3], h[3], hmx = 0.0, hmn = 1e300, d2 = 0.0;
        for (int a = 0; a < D; ++a) {
          lo[a] = g.xv[a][c[a]];
          h[a] = g.xv[a][c[a] + 1] - lo[a];
          hmx = fmax(hmx, h[a]);
          hmn = fmin(hmn, h[a]);
          d2 += h[a] * h[a];
        }
        amax = fmax(amax, hmx / hmn);
        amin = fmin(amin, hmx / hmn);
        diag += sqrt(d2);
        ++ncell;
        for (int q = 0; q < (D == 3 ? 27 : 9); ++q) {
          const int qt[3] = {q % 3, (q / 3) % 3, q / 9};
          double x[3] = {0, 0, 0};
          for (int a = 0; a < D; ++a) x[a] = lo[a] + h[a] * (qt[a] == 0 ? 0.5 - gx : (qt[a] == 1 ? 0.5 : 0.5 + gx));
          const double eta = viscosity_at(C, D, x);
          emin = fmin(emin, eta);
          emax = fmax(emax, eta);
          lsum += log10(eta);
          ++nq;
        }
      }
  // box nodes J = q v - q + a, a in [0, 2q] per axis (5^d on Q2-Q1, 3^d on Q1-Q1)
  const int ext = 2 * g.q + 1, last = (int)g.M - 1;
  int nbox = 1;
  for (int d = 0; d < D; ++d) nbox *= ext;
  int nin = 0, nbnd = 0, nvalid = 0;
  for (int m = 0; m < nbox; ++m) {
    bool in = true, bnd = false;
    int mm = m;
    for (int d = 0; d < D; ++d) {
      const int J = g.q * v[d] - g.q + mm % ext;
      mm /= ext;
      in &= (J >= 0) & (J <= last);
      bnd |= (J == 0) | (J == last);
    }
    nin += in;
    nbnd += in && bnd;
    nvalid += in && !bnd;
  }
  float* f = F + p * kF;
  f[0] = (float)log10(emax / emin);
  f[1] = (float)(lsum / nq);
  f[2] = (float)log10(amax);
  f[3] = (float)log10(amin);
  f[4] = nlev > 1 ? (float)level / (float)(nlev - 1) : 0.0f;
  f[5] = (float)(D * nvalid + 1) / (float)(D * nbox + 1);
  f[6] = nin ? (float)nbnd / (float)nin : 0.0f;
  f[7] = (float)log10(diag / ncell);
}

// ---------------------------------------------------------------------------
// Line-search labels.  One warp per subdomain: L c_i on the free rows equals
// sum_j c_j (row j of L) over the owned DoFs j (L is symmetric on the free
// DoFs), accumulated in shared memory on the local window the owned rows
// reach: Q2-Q1 nodes [2v-2, 2v+3]^d (all components) and vertices
// [v-1, v+2]^d; Q1-Q1 vertices [v-1, v+1]^d for velocity and pressure.
template <int D>
struct Win {
  static constexpr int W = 6, WV = 4;  // the Q2-Q1 extents, which bound the Q1-Q1 ones
  static constexpr int NNODE = D == 2 ? 36 : 216, NVERT = D == 2 ? 16 : 64;
  static constexpr int NLOC = D * NNODE + NVERT;
};
__device__ __forceinline__ int win_w(const Geo& g) { return g.q == 2 ? 6 : 3; }
__device__ __forceinline__ int win_wv(const Geo& g) { return g.q == 2 ? 4 : 3; }

template <int D>
__device__ __forceinline__ int win_index(const Geo& g, const int* v, int64_t m) {
  using Wn = Win<D>;
  const int W = win_w(g), WV = win_wv(g);
  if (m < g.n_u) {
    int64_t id = m / D;
    const int c = (int)(m - id * D);
    int loc = 0, mul = 1;
    for (int a = 0; a < D; ++a) {
      const int J = (int)(id % g.M);
      id /= g.M;
      const int o = J - (g.q * v[a] - g.q);
      if (o < 0 || o >= W) return -1;
      loc += o * mul;
      mul *= W;
    }
    return loc * D + c;
  }
  int64_t id = m - g.n_u;
  int loc = 0, mul = 1;
  for (int a = 0; a < D; ++a) {
    const int V = (int)(id % (g.N + 1));
    id /= (g.N + 1);
    const int o = V - (v[a] - 1);
    if (o < 0 || o >= WV) return -1;
    loc += o * mul;
    mul *= WV;
  }
  return D * Wn::NNODE + loc;
}

template <int D>
__device__ __forceinline__ int64_t win_dof(const Geo& g, const int* v, int loc) {
  using Wn = Win<D>;
  const int W = win_w(g), WV = win_wv(g);
  if (loc < D * Wn::NNODE) {
    const int c = loc % D;
    int n = loc / D;
    int64_t J[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
      J[a] = g.q * v[a] - g.q + n % W;
      n /= W;
      if (J[a] < 0 || J[a] > g.M - 1) return -1;
    }
    return D * node_id(g, J) + c;
  }
  int n = loc - D * Wn::NNODE;
  int64_t V[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) {
    V[a] = v[a] - 1 + n % WV;
    n /= WV;
    if (V[a] < 0 || V[a] > g.N) return -1;
  }
  return g.n_u + vert_id(g, V);
}

// r: the residual after the whole step, r' = r - L s; label = omega_i +
// <r', L c_i> / <L c_i, L c_i> (coordinate line search of the additive step).
template <int D>
__global__ void k_labels(Geo g, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const double* __restrict__ va, const double* __restrict__ r,
                         const double* __restrict__ c, const double* __restrict__ base, double* __restrict__ lsum,
                         int* __restrict__ lcnt) {
  using Wn = Win<D>;
  constexpr int WPB = 4;
  __shared__ double buf[WPB][Wn::NLOC];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = blockIdx.x * (int64_t)WPB + wi;
  if (p >= g.n_p) return;
  int v[3] = {0, 0, 0};
  vertex_of(g, p, v);
  for (int k = lane; k < Wn::NLOC; k += 32) buf[wi][k] = 0.0;
  __syncwarp();
  // owned DoFs: nodes 2v + delta (Q2-Q1) or vertex v itself (Q1-Q1), interior
  // ones only, all components, and p_v
  const int nr = (g.q == 2 ? (1 << D) : 1) * D + 1;
  for (int j = 0; j < nr; ++j) {
    int64_t dof;
    if (j == nr - 1) {
      dof = g.n_u + p;
    } else {
      const int q = j / D;
      int64_t J[3] = {0, 0, 0};
      bool ok = true;
      for (int d = 0; d < D; ++d) {
        J[d] = g.q == 2 ? 2 * v[d] + ((q >> d) & 1) : v[d];
        ok &= (J[d] >= 1) & (J[d] <= g.M - 2);
      }
      if (!ok) continue;
      dof = D * node_id(g, J) + j % D;
    }
    const double cj = c[dof];
    if (cj == 0.0) continue;
    for (int64_t k = rp[dof] + lane; k < rp[dof + 1]; k += 32) {
      const int64_t m = ci[k];
      if (is_dirichlet(g, m)) continue;
      const int loc = win_index<D>(g, v, m);
      if (loc >= 0) atomicAdd(&buf[wi][loc], cj * va[k]);
    }
  }
  __syncwarp();
  double num = 0.0, den = 0.0;
  for (int k = lane; k < Wn::NLOC; k += 32) {
    const double lc = buf[wi][k];
    if (lc == 0.0) continue;
    const int64_t m = win_dof<D>(g, v, k);
    num += r[m] * lc;
    den += lc * lc;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if (lane == 0) {
    double w = den > 0.0 ? base[p] + num / den : base[p];
    w = w < 0.0 ? 0.0 : (w > 1.5 ? 1.5 : w);
    lsum[p] += w;
    lcnt[p] += 1;
  }
}

__global__ void k_label_mean(int64_t np, const double* __restrict__ lsum, const int* __restrict__ lcnt,
                             double fallback, float* __restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < np) out[p] = (float)(lcnt[p] ? lsum[p] / lcnt[p] : fallback);
}

// ---------------------------------------------------------------------------
// MLP inference: fp16 weights in shared memory, fp32 accumulation; one thread
// per sample.  out_f (float) and/or out_d (double) receive omega.
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X,
                                                     int64_t n, float* __restrict__ out_f,
                                                     double* __restrict__ out_d) {
  __shared__ __half w[kNParam];
  for (int i = threadIdx.x; i < kNParam; i += blockDim.x) w[i] = __float2half_rn(P[i]);
  __syncthreads();
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const __half *W1 = w, *b1 = W1 + kH * kF, *W2 = b1 + kH, *b2 = W2 + kH * kH, *W3 = b2 + kH, *b3 = W3 + kH;
  float f[kF], a1[kH];
#pragma unroll
  for (int k = 0; k < kF; ++k) f[k] = X[s * kF + k];
#pragma unroll 4
  for (int i = 0; i < kH; ++i) {
    float t = __half2float(b1[i]);
#pragma unroll
    for (int k = 0; k < kF; ++k) t += __half2float(W1[i * kF + k]) * f[k];
    a1[i] = t > 0.0f ? t : 0.0f;
  }
  float z = __half2float(b3[0]);
  for (int i = 0; i < kH; ++i) {
    float t = __half2float(b2[i]);
#pragma unroll 8
    for (int k = 0; k < kH; ++k) t += __half2float(W2[i * kH + k]) * a1[k];
    z += __half2float(W3[i]) * (t > 0.0f ? t : 0.0f);
  }
  const float om = 1.5f / (1.0f + expf(-z));
  if (out_f) out_f[s] = om;
  if (out_d) out_d[s] = (double)om;
}

// MLP training gradient (fp32 weights): one block of TB samples computes its
// samples' activations and deltas in shared memory, then its share of every
// parameter's gradient; partials per block, summed by k_grad_reduce.
constexpr int TB = 64;
__global__ void __launch_bounds__(128) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                  const float* __restrict__ y, int64_t n, float inv_n,
                                                  float* __restrict__ part, float* __restrict__ part_loss) {
  extern __shared__ float sm[];
  float* w = sm;                    // kNParam
  float* A1 = w + kNParam;          // TB x kH
  float* A2 = A1 + TB * kH;         // TB x kH
  float* D1 = A2 + TB * kH;         // TB x kH
  float* D2 = D1 + TB * kH;         // TB x kH
  float* FX = D2 + TB * kH;         // TB x kF
  float* DZ = FX + TB * kF;         // TB
  for (int i = threadIdx.x; i < kNParam; i += blockDim.x) w[i] = P[i];
  const int64_t s0 = blockIdx.x * (int64_t)TB;
  const int ns = (int)(n - s0 < TB ? n - s0 : TB);
  for (int i = threadIdx.x; i < TB * kF; i += blockDim.x) {
    const int s = i / kF;
    FX[i] = s < ns ? X[(s0 + s) * kF + i % kF] : 0.0f;
  }
  __syncthreads();
  const float *W1 = w, *b1 = W1 + kH * kF, *W2 = b1 + kH, *b2 = W2 + kH * kH, *W3 = b2 + kH, *b3 = W3 + kH;
  // layer 1: thread t handles (sample, unit) pairs
  for (int e = threadIdx.x; e < TB * kH; e += blockDim.x) {
    const int s = e / kH, i = e % kH;
    float t = b1[i];
    for (int k = 0; k < kF; ++k) t += W1[i * kF + k] * FX[s * kF + k];
    A1[e] = t > 0.0f ? t : 0.0f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TB * kH; e += blockDim.x) {
    const int s = e / kH, i = e % kH;
    float t = b2[i];
    for (int k = 0; k < kH; ++k) t += W2[i * kH + k] * A1[s * kH + k];
    A2[e] = t > 0.0f ? t : 0.0f;
  }
  __syncthreads();
  float lsum = 0.0f;
  for (int s = threadIdx.x; s < TB; s += blockDim.x) {
    float z = b3[0];
    for (int k = 0; k < kH; ++k) z += W3[k] * A2[s * kH + k];
    const float sg = 1.0f / (1.0f + expf(-z));
    const float e = 1.5f * sg - (s < ns ? y[s0 + s] : 0.0f);
    DZ[s] = s < ns ? 2.0f * e * inv_n * 1.5f * sg * (1.0f - sg) : 0.0f;
    lsum += s < ns ? e * e * inv_n : 0.0f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TB * kH; e += blockDim.x) {
    const int s = e / kH, k = e % kH;
    D2[e] = A2[e] > 0.0f ? DZ[s] * W3[k] : 0.0f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TB * kH; e += blockDim.x) {
    const int s = e / kH, k = e % kH;
    float t = 0.0f;
    for (int i = 0; i < kH; ++i) t += W2[i * kH + k] * D2[s * kH + i];
    D1[e] = A1[e] > 0.0f ? t : 0.0f;
  }
  __syncthreads();
  float* g = part + blockIdx.x * (int64_t)kNParam;
  float *gW1 = g, *gb1 = gW1 + kH * kF, *gW2 = gb1 + kH, *gb2 = gW2 + kH * kH, *gW3 = gb2 + kH, *gb3 = gW3 + kH;
  for (int e = threadIdx.x; e < kH * kH; e += blockDim.x) {
    const int i = e / kH, k = e % kH;
    float t = 0.0f;
    for (int s = 0; s < TB; ++s) t += D2[s * kH + i] * A1[s * kH + k];
    gW2[e] = t;
  }
  for (int e = threadIdx.x; e < kH * kF; e += blockDim.x) {
    const int i = e / kF, k = e % kF;
    float t = 0.0f;
    for (int s = 0; s < TB; ++s) t += D1[s * kH + i] * FX[s * kF + k];
    gW1[e] = t;
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    float t1 = 0.0f, t2 = 0.0f, t3 = 0.0f;
    for (int s = 0; s < TB; ++s) {
      t1 += D1[s * kH + i];
      t2 += D2[s * kH + i];
      t3 += DZ[s] * A2[s * kH + i];
    }
    gb1[i] = t1;
    gb2[i] = t2;
    gW3[i] = t3;
  }
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int s = 0; s < TB; ++s) t += DZ[s];
    gb3[0] = t;
  }
  // loss partial
  __shared__ float red[128];
  red[threadIdx.x] = lsum;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part_loss[blockIdx.x] = red[0];
}

__global__ void k_grad_reduce(const float* __restrict__ part, const float* __restrict__ part_loss, int nb,
                              float* __restrict__ grad, float* __restrict__ loss) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < kNParam) {
    float t = 0.0f;
    for (int b = 0; b < nb; ++b) t += part[(int64_t)b * kNParam + j];
    grad[j] = t;
  }
  if (j == 0 && loss) {
    float t = 0.0f;
    for (int b = 0; b < nb; ++b) t += part_loss[b];
    *loss = t;
  }
}

__global__ void k_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kNParam) return;
  const float gj = g[j];
  const float mj = b1 * m[j] + (1.0f - b1) * gj;
  const float vj = b2 * v[j] + (1.0f - b2) * gj * gj;
  m[j] = mj;
  v[j] = vj;
  P[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
}

}  // namespace rav

using namespace rav;

extern "C" int rav_mlp_nparam(void) { return kNParam; }

extern "C" int rav_patch_features(rav_smoother* sm, int level, float* feat, rav_stream stream) {
  if (!sm || !feat || level < 1 || level >= sm->mg->nlev) return RAV_ERR_ARG;
  rav_mg* mg = sm->mg;
  const Geo& g = mg->lev[level].g;
  Coef C{mg->eta0, mg->nblobs, mg->blobs_dev};
  const int blocks = (int)((g.n_p + 127) / 128);
  if (g.dim == 2) k_features<2><<<blocks, 128, 0, S(stream)>>>(g, C, level, mg->nlev, feat);
  else k_features<3><<<blocks, 128, 0, S(stream)>>>(g, C, level, mg->nlev, feat);
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

extern "C" int rav_label_collection(rav_smoother* sm, int enable) {
  if (!sm) return RAV_ERR_ARG;
  if (sm->kind != RAV_RAV) return RAV_ERR_ARG;
  rav_mg* mg = sm->mg;
  sm->collect = enable != 0;
  if (!sm->collect) return RAV_OK;
  drop_graphs(mg, sm);
  for (int l = 1; l < mg->nlev; ++l) {
    SmLevel& SL = sm->lev[l];
    const int64_t np = SL.np, n = mg->lev[l].g.n;
    if (!SL.lsum) {
      RAV_CUDA(cudaMalloc(&SL.lsum, sizeof(double) * np));
      RAV_CUDA(cudaMalloc(&SL.lcnt, sizeof(int) * np));
      RAV_CUDA(cudaMalloc(&SL.ones, sizeof(double) * np));
      RAV_CUDA(cudaMalloc(&SL.ctmp, sizeof(double) * n));
      RAV_CUDA(cudaMalloc(&SL.stmp, sizeof(double) * n));
      RAV_CUDA(cudaMalloc(&SL.rtmp, sizeof(double) * n));
      std::vector<double> one(np, 1.0);
      RAV_CUDA(cudaMemcpy(SL.ones, one.data(), sizeof(double) * np, cudaMemcpyHostToDevice));
    }
    RAV_CUDA(cudaMemset(SL.lsum, 0, sizeof(double) * np));
    RAV_CUDA(cudaMemset(SL.lcnt, 0, sizeof(int) * np));
  }
  return RAV_OK;
}

// Called by the smoother, before its apply, while collection is on: c = the
// subdomains' own corrections (weight 1) for residual r, s = the whole step
// with the current weights, r' = r - L s, then the labels.
int collect_labels(rav_smoother* sm, int level, const double* r, cudaStream_t s) {
  rav_mg* mg = sm->mg;
  SmLevel& SL = sm->lev[level];
  Level& L = mg->lev[level];
  RAV_CUDA(cudaMemsetAsync(SL.ctmp, 0, sizeof(double) * L.g.n, s));
  RAV_CUDA(cudaMemsetAsync(SL.stmp, 0, sizeof(double) * L.g.n, s));
  RAV_TRY(apply_with_omega(sm, level, r, SL.ctmp, SL.ones, s));
  RAV_TRY(apply_with_omega(sm, level, r, SL.stmp, SL.omega, s));
  RAV_TRY(residual_impl(mg, level, SL.stmp, r, SL.rtmp, nullptr, s));
  const unsigned gb = (unsigned)((L.g.n_p + 3) / 4);
  if (L.g.dim == 2)
    k_labels<2><<<gb, 128, 0, s>>>(L.g, L.rp, L.ci, L.va, SL.rtmp, SL.ctmp, SL.omega, SL.lsum, SL.lcnt);
  else
    k_labels<3><<<gb, 128, 0, s>>>(L.g, L.rp, L.ci, L.va, SL.rtmp, SL.ctmp, SL.omega, SL.lsum, SL.lcnt);
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

extern "C" int rav_read_labels(rav_smoother* sm, int level, float* out, rav_stream stream) {
  if (!sm || !out || level < 1 || level >= sm->mg->nlev || !sm->lev[level].lsum) return RAV_ERR_ARG;
  const SmLevel& SL = sm->lev[level];
  k_label_mean<<<(int)((SL.np + 255) / 256), 256, 0, S(stream)>>>(SL.np, SL.lsum, SL.lcnt, sm->omega, out);
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

extern "C" int rav_mlp_forward(const float* params, const float* X, int64_t n, float* omega, rav_stream stream) {
  if (!params || !X || !omega || n < 0) return RAV_ERR_ARG;
  if (n == 0) return RAV_OK;
  k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, S(stream)>>>(params, X, n, omega, nullptr);
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

extern "C" int rav_mlp_loss_grad(const float* params, const float* X, const float* y, int64_t n, float* grad,
                                 float* loss, float* work, int64_t work_floats, rav_stream stream) {
  if (!params || !X || !y || !grad || n <= 0) return RAV_ERR_ARG;
  const int64_t nb = (n + TB - 1) / TB;
  if (!work || work_floats < nb * (kNParam + 1)) return RAV_ERR_ARG;
  cudaStream_t s = S(stream);
  const size_t smem = sizeof(float) * (kNParam + 4 * TB * kH + TB * kF + TB);
  RAV_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  float* part = work;
  float* part_loss = work + nb * kNParam;
  k_mlp_grad<<<(unsigned)nb, 128, smem, s>>>(params, X, y, n, 1.0f / (float)n, part, part_loss);
  k_grad_reduce<<<(kNParam + 255) / 256, 256, 0, s>>>(part, part_loss, (int)nb, grad, loss);
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

extern "C" int rav_adam_step(float* params, float* m, float* v, const float* grad, float lr, int t,
                             rav_stream stream) {
  if (!params || !m || !v || !grad || t < 1) return RAV_ERR_ARG;
  const float b1 = 0.9f, b2 = 0.999f;
  k_adam<<<(kNParam + 255) / 256, 256, 0, S(stream)>>>(params, m, v, grad, lr, b1, b2, 1e-8f,
                                                       1.0f - powf(b1, (float)t), 1.0f - powf(b2, (float)t));
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

// omega_i <- m + shrink * (omega_i - m), m the mean over the level (one block).
__global__ void k_shrink_to_mean(double* __restrict__ w, int64_t n, double shrink) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += w[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double m = red[0] / (double)n;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) w[i] = m + shrink * (w[i] - m);
}

extern "C" int rav_set_learned_omega(rav_smoother* sm, const float* params, double shrink, rav_stream stream) {
  if (!sm || !params || !(shrink >= 0.0 && shrink <= 1.0)) return RAV_ERR_ARG;
  rav_mg* mg = sm->mg;
  cudaStream_t s = S(stream);
  for (int l = 1; l < mg->nlev; ++l) {
    const int64_t np = sm->lev[l].np;
    float* feat = nullptr;
    RAV_CUDA(cudaMallocAsync(&feat, sizeof(float) * np * kF, s));
    const int rc = rav_patch_features(sm, l, feat, stream);
    if (rc == RAV_OK) {
      k_mlp_forward<<<(unsigned)((np + 127) / 128), 128, 0, s>>>(params, feat, np, nullptr, sm->lev[l].omega);
      if (shrink < 1.0) k_shrink_to_mean<<<1, 1024, 0, s>>>(sm->lev[l].omega, np, shrink);
    }
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(feat, s);
    if (rc != RAV_OK) return rc;
    RAV_CUDA(e);
  }
  return RAV_OK;
}

extern "C" int rav_reset_omega(rav_smoother* sm, rav_stream stream) {
  if (!sm) return RAV_ERR_ARG;
  return reset_omega(sm, S(stream));
}
