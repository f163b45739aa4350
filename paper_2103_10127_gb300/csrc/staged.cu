// Staged subdomain apply for the reduced factored storage (RAV_F32_FACT,
// RAV_BF16_FACT) on Q2-Q1 levels.
//
// It computes Eq. 13 through the block form of L_i^{-1} (one pressure DoF per
// subdomain, A_i = I_d (x) K_i):
//   tau = (1/s) (w^T r_u - r_p),
//   y(m,c) = sum_n K^{-1}[m,n] r(n,c) + w(m,c) tau   for the owned nodes m,
//   y_p = -tau,   x[owned] += omega_i y,
// the same arithmetic as k_rav_apply_fact, laid out for streaming:
//
// * Gather (the patch restriction R_i r of Sec. 3).  A thread block owns a
//   tile of TX x TY (x TZ) vertices.  The boxes of its subdomains cover the Q2
//   nodes 2 v0 - 2 ... 2 (v0 + T) per axis, (2T+3) per axis, which the block
//   copies once from the fp32 residual into shared memory (zero outside the
//   domain; r is zero on Dirichlet rows already), so every box read is a
//   shared-memory load with no bounds test and no global address arithmetic.
// * Local solve.  S threads per subdomain; split s takes the box nodes
//   n = s, s + S, ... and, per node, multiplies the 2^d owned rows of K^{-1}
//   with the d residual components (2^d d FMAs) and adds its share of w^T r_u
//   (d FMAs); the S partial sums meet by shuffles.  Products accumulate in
//   fp32 from the fp32-rounded residual, as in the other reduced applies.
// * Restricted scatter (Eq. 13).  The owned DoFs of different subdomains are
//   disjoint: plain fp64 read-modify-writes of x, no atomics.
// * Streaming.  Thread slot k = l S + s of tile t (l = subdomain of the tile,
//   x fastest) reads at node step j the chunk ((t NJ + j) W + k / 32) 32 + k % 32
//   (W warps per tile, NJ = ceil(5^d / S) steps), holding the 2^d values
//   K^{-1}[q, n], q = 0 .. 2^d - 1, and in a second array the d values
//   w(n, c) (zero padded to WC), n = s + S j (zero chunks past the last box
//   node), so the threads of a block read one contiguous run per step.  Each
//   thread keeps kStRing steps of its chunks in flight in registers.  1/s per
//   subdomain slot.  The chunks are rebuilt from the grouped factored
//   storage (k_restage), so they hold exactly the same rounded values.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <type_traits>

#include "box.cuh"
#include "common.cuh"
#include "cpasync.cuh"
#include "fmt.cuh"

namespace rav {

template <int D>
struct StagedBox {
  static constexpr int NV = BoxT<D>::NV;    // box nodes
  static constexpr int NON = BoxT<D>::NON;  // owned nodes
  static constexpr int WC = D == 3 ? 4 : 2; // w values per chunk (3-D: 3 and a zero)
};

// Streaming of the chunks: every thread keeps kStRing node steps of its own
// chunks in flight in registers (evict-first loads; the loop is unrolled by
// kStRing so that every slot is known at compile time).
constexpr int kStRing = 4;

// Shared-memory plan of a block of nthr threads: the epilogue slots (per
// thread the x values and w chunks of the owned nodes it writes, fetched at
// the start), the staged residual nodes, the box-node offset table.
template <int D, typename T, int S>
struct StagedPlan {
  static constexpr int NV = StagedBox<D>::NV, NON = StagedBox<D>::NON, WC = StagedBox<D>::WC;
  static constexpr int NJ = (NV + S - 1) / S;
  static constexpr int CK = NON * (int)sizeof(T), CW = WC * (int)sizeof(T);
  static constexpr int OWN = (NON + S - 1) / S;              // owned nodes written per thread
  static constexpr int OFFX = (CW + 7) / 8 * 8;               // per owned node: its w chunk, then
  static constexpr int BLK = (OFFX + 8 * D + 15) / 16 * 16;   // its d fp64 x values (16-byte blocks)
  static constexpr int EPI = OWN * BLK;
  __host__ __device__ static size_t epi_off(int) { return 0; }
  __host__ __device__ static size_t nodes_off(int nthr) { return epi_off(nthr) + (size_t)EPI * nthr; }
  __host__ __device__ static size_t offs_off(const StagedGeo& sg) {
    return nodes_off(sg.wpt * 32) + (size_t)sg.sx * sg.sy * sg.sz * (D == 3 ? 16 : 8);
  }
  __host__ __device__ static size_t bytes(const StagedGeo& sg) { return offs_off(sg) + sizeof(int) * NJ * S; }
};

// Launch bounds: 3 blocks of 256 threads per SM (85 registers: the
// accumulators and kStRing chunks in flight); 3-D fp32 chunks are twice as
// large and run in blocks of at most 128 threads, 4 per SM (128 registers).
template <int D, typename T>
constexpr int staged_max_threads() {
  return (D == 3 && sizeof(T) == 4) ? 128 : 256;
}
template <int D, typename T>
constexpr int staged_min_blocks() {
  return (D == 3 && sizeof(T) == 4) ? 4 : 3;
}

template <int D, typename T, int S>
__global__ void __launch_bounds__(staged_max_threads<D, T>(), staged_min_blocks<D, T>()) k_rav_apply_staged(Geo g, StagedGeo sg, const T* __restrict__ kq,
                                                            const T* __restrict__ wq, const float* __restrict__ sinv,
                                                            const double* __restrict__ omega,
                                                            const float* __restrict__ r32, double* __restrict__ x) {
  using P = StagedPlan<D, T, S>;
  using RV = typename NodeT<D>::type;
  constexpr int NV = P::NV, NON = P::NON, WC = P::WC, NJ = P::NJ, CK = P::CK, CW = P::CW;
  extern __shared__ __align__(128) uint8_t sraw[];
  const int nthr = sg.wpt * 32;
  const int tid = threadIdx.x;
  uint8_t* epi = sraw + P::epi_off(nthr) + (size_t)tid * P::EPI;
  RV* tile = reinterpret_cast<RV*>(sraw + P::nodes_off(nthr));
  int* offs = reinterpret_cast<int*>(sraw + P::offs_off(sg));
  const int nst = sg.sx * sg.sy * (D == 3 ? sg.sz : 1);
  const int t = blockIdx.x;
  const int l = tid / S, s = tid % S;
  const int TS = sg.tx * sg.ty * sg.tz;
  const int tix = t % sg.ntx, tiy = (t / sg.ntx) % sg.nty, tiz = D == 3 ? t / (sg.ntx * sg.nty) : 0;
  const int v0x = tix * sg.tx, v0y = tiy * sg.ty, v0z = tiz * sg.tz;
  const int lx = l % sg.tx, ly = (l / sg.tx) % sg.ty, lz = D == 3 ? l / (sg.tx * sg.ty) : 0;
  const int v[3] = {v0x + lx, v0y + ly, v0z + lz};
  // threads of slots outside the grid (or past the tile) only help staging r
  const bool active = l < TS && v[0] <= g.N && v[1] <= g.N && (D == 2 || v[2] <= g.N);
  const size_t cstride = (size_t)nthr;  // chunks per node step of the block
  // group 0: the tile's residual boxes (every thread a share, zero outside the
  // domain; r is zero on Dirichlet rows already) and this thread's epilogue data
  const int64_t M = g.M;
  for (int i = tid; i < nst; i += blockDim.x) {
    const int i0 = i % sg.sx, i1 = (i / sg.sx) % sg.sy, i2 = D == 3 ? i / (sg.sx * sg.sy) : 0;
    const int64_t J0 = 2 * v0x - 2 + i0, J1 = 2 * v0y - 2 + i1, J2 = D == 3 ? 2 * v0z - 2 + i2 : 0;
    bool in = J0 >= 0 && J0 < M && J1 >= 0 && J1 < M;
    if (D == 3) in = in && J2 >= 0 && J2 < M;
    const float* src = r32 + (in ? (J0 + M * (J1 + M * J2)) * D : 0);
    float* dst = reinterpret_cast<float*>(tile + i);
#pragma unroll
    for (int c = 0; c < D; ++c) st_copy4z(dst + c, src + c, in);
    if (D == 3) dst[3] = 0.f;
  }
  // owned node q (bit d = offset on axis d) is written by split q % S: its first
  // velocity DoF (-1: a Dirichlet node) and its box position mq
  auto owned = [&](int q, int& mq) -> int64_t {
    int64_t J[3] = {0, 0, 0};
    bool ok = true;
    mq = 0;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) {
      const int dl = (q >> d) & 1;
      J[d] = 2 * v[d] + dl;
      ok &= (J[d] >= 1) & (J[d] <= 2 * g.N - 1);
      mq = mq * 5 + 2 + dl;
    }
    return ok ? D * node_id_t<D>(g, J) : -1;
  };
  if (active) {
#pragma unroll
    for (int k = 0; k < P::OWN; ++k) {
      const int q = s + S * k;
      if (q >= NON) continue;
      int mq;
      const int64_t dof = owned(q, mq);
      if (dof < 0) continue;
      double* ex = reinterpret_cast<double*>(epi + k * P::BLK + P::OFFX);
#pragma unroll
      for (int c = 0; c < D; ++c) st_copy<8>(ex + c, x + dof + c);
      // w at the owned node's box position: its chunk, streamed by split mq % S at step mq / S
      const int kk = l * S + mq % S;
      const size_t ci = ((size_t)t * NJ + mq / S) * cstride + kk;
      st_copy<CW>(epi + k * P::BLK, wq + ci * WC);
    }
  }
  st_commit();
  // the first node steps of this thread's chunk stream, in flight while the tile lands
  const T* kme = kq + ((size_t)t * NJ * cstride + tid) * NON;
  const T* wme = wq + ((size_t)t * NJ * cstride + tid) * WC;
  constexpr int R = kStRing;
  RawChunk<CK> kb[R];
  RawChunk<CW> wb[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    if (active && j < NJ) {
      kb[j] = ld_raw<CK>(kme + (size_t)j * cstride * NON);
      wb[j] = ld_raw<CW>(wme + (size_t)j * cstride * WC);
    } else {
#pragma unroll
      for (int i = 0; i < CK / 4; ++i) kb[j].w[i] = 0u;
#pragma unroll
      for (int i = 0; i < CW / 4; ++i) wb[j].w[i] = 0u;
    }
  }
  for (int n = tid; n < NJ * S; n += blockDim.x) {
    int off = 0;  // padded node: any staged node (its stored values are zero)
    if (n < NV) {
      const int a0 = n % 5, a1 = (n / 5) % 5, a2 = D == 3 ? n / 25 : 0;
      off = a0 + sg.sx * (a1 + sg.sy * a2);
    }
    offs[n] = off;
  }
  st_wait<0>();  // group 0 has landed
  __syncthreads();
  if (!active) return;
  const int base = ((D == 3 ? 2 * lz * sg.sy : 0) + 2 * ly) * sg.sx + 2 * lx;
  float y[NON][D], tw = 0.f;
#pragma unroll
  for (int q = 0; q < NON; ++q)
#pragma unroll
    for (int c = 0; c < D; ++c) y[q][c] = 0.f;
#pragma unroll 1
  for (int j0 = 0; j0 < NJ; j0 += R) {
#pragma unroll
    for (int q = 0; q < R; ++q) {  // slot q holds step j = j0 + q
      const int j = j0 + q;
      if (j < NJ) {
        float kf[NON], wf[WC];
        widen_words<T, CK / 4>(kb[q].w, kf);
        widen_words<T, CW / 4>(wb[q].w, wf);
        const RV rv = tile[base + offs[s + S * j]];
        float rc[D];
        rc[0] = rv.x;
        rc[1] = rv.y;
        if constexpr (D == 3) rc[2] = reinterpret_cast<const float4&>(rv).z;
#pragma unroll
        for (int qq = 0; qq < NON; ++qq)
#pragma unroll
          for (int c = 0; c < D; ++c) y[qq][c] = fmaf(kf[qq], rc[c], y[qq][c]);
#pragma unroll
        for (int c = 0; c < D; ++c) tw = fmaf(wf[c], rc[c], tw);
        // the slot is read (its values are in the FMAs above): refill it with step j + R
        if (j + R < NJ) {
          kb[q] = ld_raw<CK>(kme + (size_t)(j + R) * cstride * NON);
          wb[q] = ld_raw<CW>(wme + (size_t)(j + R) * cstride * WC);
        }
      }
    }
  }
  const int lane = tid & 31;
  const unsigned gmask = S == 32 ? 0xffffffffu : (((1u << S) - 1u) << (lane & ~(S - 1)));
#pragma unroll
  for (int o = 1; o < S; o <<= 1) {
#pragma unroll
    for (int q = 0; q < NON; ++q)
#pragma unroll
      for (int c = 0; c < D; ++c) y[q][c] += __shfl_xor_sync(gmask, y[q][c], o);
    tw += __shfl_xor_sync(gmask, tw, o);
  }
  const int64_t p = v[0] + (int64_t)(g.N + 1) * (v[1] + (int64_t)(g.N + 1) * v[2]);
  const float tau = sinv[(int64_t)t * TS + l] * (tw - r32[g.n_u + p]);
  const double om = omega[p];
#pragma unroll
  for (int k = 0; k < P::OWN; ++k) {
    const int q = s + S * k;
    if (q >= NON) continue;
    int mq;
    const int64_t dof = owned(q, mq);
    if (dof < 0) continue;
    const double* ex = reinterpret_cast<const double*>(epi + k * P::BLK + P::OFFX);
    float wm[WC];
    sm_chunk<T, WC>(reinterpret_cast<const T*>(epi + k * P::BLK), wm);
    float yq[D];
#pragma unroll
    for (int c = 0; c < D; ++c) yq[c] = y[0][c];
#pragma unroll
    for (int qq = 1; qq < NON; ++qq)
      if (qq == q)
#pragma unroll
        for (int c = 0; c < D; ++c) yq[c] = y[qq][c];
#pragma unroll
    for (int c = 0; c < D; ++c) x[dof + c] = ex[c] + om * (double)(yq[c] + wm[c] * tau);
  }
  if (s == 0) x[g.n_u + p] += om * (double)-tau;
}

// Builds the staged chunks of level storage from the grouped factored storage
// (K^{-1} rows of unit u = p 2^d + q at ((u / G) NV + n) G + u % G, G = 2^lg;
// w and 1/s per subdomain, NV d + 1 values): one thread per (subdomain, box
// node chunk).  Values are copied bit for bit; 1/s is widened to fp32.
template <int D, typename T, int S>
__global__ void k_restage(Geo g, StagedGeo sg, const T* __restrict__ kinv, const T* __restrict__ ws, int lg,
                          T* __restrict__ kq, T* __restrict__ wq, float* __restrict__ sinv) {
  using SB = StagedBox<D>;
  constexpr int NV = SB::NV, NON = SB::NON, WC = SB::WC, NWS = D * NV + 1;
  constexpr int NJ = (NV + S - 1) / S;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= g.n_p * (int64_t)(NJ * S)) return;
  const int64_t p = e / (NJ * S);
  const int n = (int)(e % (NJ * S));
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  const int t = v[0] / sg.tx + sg.ntx * (v[1] / sg.ty + sg.nty * (D == 3 ? v[2] / sg.tz : 0));
  const int l = v[0] % sg.tx + sg.tx * (v[1] % sg.ty + sg.ty * (D == 3 ? v[2] % sg.tz : 0));
  const int s = n % S, j = n / S;
  const int k = l * S + s;
  const int64_t ci = (((int64_t)t * NJ + j) * sg.wpt + (k >> 5)) * 32 + (k & 31);
  const int64_t G = int64_t(1) << lg;
  const T zero = Fmt<T>::enc(0.0);
#pragma unroll
  for (int q = 0; q < NON; ++q) {
    const int64_t u = p * NON + q;
    kq[ci * NON + q] = n < NV ? kinv[((u >> lg) * NV + n) * G + (u & (G - 1))] : zero;
  }
#pragma unroll
  for (int c = 0; c < WC; ++c) wq[ci * WC + c] = (n < NV && c < D) ? ws[p * NWS + n * D + c] : zero;
  if (n == 0) sinv[(int64_t)t * (sg.tx * sg.ty * sg.tz) + l] = Fmt<T>::dec(ws[p * NWS + NWS - 1], nullptr);
}

}  // namespace rav

using namespace rav;

// Tiles of vertices for a level of N cells per axis and S threads per
// subdomain: 64 to max_threads threads per block and at most 100 KiB of shared
// memory (epilogue slots: epi_per_warp bytes per warp, plus the staged residual
// nodes).  Candidates are ranked by idle thread slots (tiles past the grid's
// last vertex) and the use of the last wave, with a penalty for halo (staged
// nodes per owned node); per_sm_of(threads, shared bytes) gives a candidate's
// resident blocks per SM (the kernel's registers, shared memory and threads),
// nsm the SM count.  cand picks the cand-th best of distinct block counts (the
// set-up tuner times the first few).  tx == 0: no candidate.
StagedGeo staged_tiles(int D, int N, int S, size_t epi_per_warp, int max_threads, int cand,
                       const std::function<int(int, size_t)>& per_sm_of, int nsm) {
  const int mv = N + 1;
  struct Cand {
    double score;
    StagedGeo sg;
  };
  std::vector<Cand> all;
  const int zmax = D == 3 ? std::min(mv, 16) : 1;
  for (int tx = 1; tx <= std::min(mv, 64); ++tx)
    for (int ty = 1; ty <= std::min(mv, 32); ++ty)
      for (int tz = 1; tz <= zmax; ++tz) {
        const int ts = tx * ty * tz, thr = ts * S;
        if (thr > max_threads || thr < std::min(64, (D == 3 ? mv * mv * mv : mv * mv) * S)) continue;
        const int ntx = (mv + tx - 1) / tx, nty = (mv + ty - 1) / ty, ntz = D == 3 ? (mv + tz - 1) / tz : 1;
        const double tiles = (double)ntx * nty * ntz;
        const int wpt = (thr + 31) / 32;
        const double slots = tiles * wpt * 32;
        const double used = (D == 3 ? (double)mv * mv * mv : (double)mv * mv) * S;
        const double nodes = (2.0 * tx + 3) * (2.0 * ty + 3) * (D == 3 ? 2.0 * tz + 3 : 1.0);
        const double smem = nodes * (D == 3 ? 16 : 8) + (double)epi_per_warp * wpt;
        if (smem > 100 * 1024) continue;
        const double halo = nodes / (ts * (D == 3 ? 8.0 : 4.0));
        // resident blocks per SM and the share of the last wave's slots used
        const int per_sm = std::max(1, per_sm_of(wpt * 32, (size_t)smem + 512));
        const double slots_gpu = (double)nsm * per_sm;
        const double wave_use = tiles / (std::ceil(tiles / slots_gpu) * slots_gpu);
        const double score = slots / used * (1.0 + 0.15 * halo) / wave_use;
        all.push_back({score, StagedGeo{tx, ty, tz, ntx, nty, ntz, wpt, 2 * tx + 3, 2 * ty + 3,
                                        D == 3 ? 2 * tz + 3 : 1}});
      }
  std::sort(all.begin(), all.end(), [](const Cand& a, const Cand& b) { return a.score < b.score; });
  std::vector<int64_t> seen;
  for (const Cand& c : all) {
    const int64_t key = (int64_t)c.sg.ntx * c.sg.nty * c.sg.ntz * 4096 + c.sg.wpt;
    if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
    if ((int)seen.size() == cand) return c.sg;
    seen.push_back(key);
  }
  return StagedGeo{};
}

// Frees the staged chunks of a level (its grouped storage stays).
void staged_free(SmLevel& SL) {
  cudaFree(SL.skq);
  cudaFree(SL.swq);
  cudaFree(SL.ssinv);
  SL.skq = SL.swq = nullptr;
  SL.ssinv = nullptr;
  SL.staged = 0;
}

template <int D, typename T, int S>
static int restage_t(const Geo& g, SmLevel& SL, int cand, cudaStream_t s) {
  using P = StagedPlan<D, T, S>;
  using SB = StagedBox<D>;
  constexpr int NJ = P::NJ;
  const int max_thr = staged_max_threads<D, T>();
  // the attribute is per kernel instance, shared by every level: allow the
  // largest plan staged_tiles admits (100 KiB and the small tables after it)
  RAV_CUDA(cudaFuncSetAttribute(k_rav_apply_staged<D, T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                104 * 1024));
  int dev = 0, nsm = 0;
  RAV_CUDA(cudaGetDevice(&dev));
  RAV_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  auto per_sm_of = [](int thr, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rav_apply_staged<D, T, S>, thr, smem) != cudaSuccess)
      return 1;
    return nb;
  };
  const StagedGeo sg = staged_tiles(D, g.N, S, (size_t)32 * P::EPI, max_thr, cand, per_sm_of, nsm);
  if (sg.tx == 0) return RAV_ERR_ARG;
  const int64_t tiles = (int64_t)sg.ntx * sg.nty * sg.ntz;
  const int64_t chunks = tiles * sg.wpt * NJ * 32;
  staged_free(SL);
  RAV_CUDA(cudaMalloc(&SL.skq, sizeof(T) * chunks * SB::NON));
  RAV_CUDA(cudaMalloc(&SL.swq, sizeof(T) * chunks * SB::WC));
  RAV_CUDA(cudaMalloc(&SL.ssinv, sizeof(float) * tiles * sg.tx * sg.ty * sg.tz));
  RAV_CUDA(cudaMemsetAsync(SL.skq, 0, sizeof(T) * chunks * SB::NON, s));
  RAV_CUDA(cudaMemsetAsync(SL.swq, 0, sizeof(T) * chunks * SB::WC, s));
  RAV_CUDA(cudaMemsetAsync(SL.ssinv, 0, sizeof(float) * tiles * sg.tx * sg.ty * sg.tz, s));
  int lg = 0;
  while ((1 << lg) < 32 / SL.split) ++lg;
  const int64_t tot = g.n_p * (int64_t)(NJ * S);
  k_restage<D, T, S><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g, sg, (const T*)SL.inv, (const T*)SL.ws, lg,
                                                                  (T*)SL.skq, (T*)SL.swq, SL.ssinv);
  RAV_CUDA(cudaGetLastError());
  if (P::bytes(sg) > 104 * 1024) return RAV_ERR_ARG;
  SL.sgeo = sg;
  SL.staged = S;
  return RAV_OK;
}

// (Re)builds the staged chunks of a reduced factored Q2-Q1 level for S threads
// per subdomain and the cand-th tiling candidate: S = 1 the streamed kernel of
// stream.cu (one tiling), 2-D S = 2, 3-D S = 2 or 4 the kernel above; S = 0
// frees them (the grouped kernel is used again).  RAV_ERR_ARG when there is no
// such candidate.
int staged_build(rav_smoother* sm, int level, int S, cudaStream_t s, int cand) {
  SmLevel& SL = sm->lev[level];
  const Geo& g = sm->mg->lev[level].g;
  if (S == 0) {
    staged_free(SL);
    return RAV_OK;
  }
  if (S == 1) return cand == 0 ? stream_build(sm, level, s) : RAV_ERR_ARG;
  const bool bf = sm->prec == RAV_BF16_FACT;
  if (g.dim == 2) {
    if (S == 2) return bf ? restage_t<2, __nv_bfloat16, 2>(g, SL, cand, s) : restage_t<2, float, 2>(g, SL, cand, s);
  } else {
    if (S == 2) return bf ? restage_t<3, __nv_bfloat16, 2>(g, SL, cand, s) : restage_t<3, float, 2>(g, SL, cand, s);
    if (S == 4) return bf ? restage_t<3, __nv_bfloat16, 4>(g, SL, cand, s) : restage_t<3, float, 4>(g, SL, cand, s);
  }
  return RAV_ERR_ARG;
}

template <int D, typename T, int S>
static void launch_staged_t(const Geo& g, const SmLevel& SL, const double* omega, const float* r32, double* x,
                            cudaStream_t s) {
  const StagedGeo& sg = SL.sgeo;
  const unsigned tiles = (unsigned)((int64_t)sg.ntx * sg.nty * sg.ntz);
  k_rav_apply_staged<D, T, S><<<tiles, sg.wpt * 32, StagedPlan<D, T, S>::bytes(sg), s>>>(
      g, sg, (const T*)SL.skq, (const T*)SL.swq, SL.ssinv, omega, r32, x);
}

// One staged apply x += S_RAV r on a level whose chunks are built.
void staged_launch(const rav_smoother* sm, int level, const double* omega, const float* r32, double* x,
                   cudaStream_t s) {
  const SmLevel& SL = sm->lev[level];
  const Geo& g = sm->mg->lev[level].g;
  if (SL.staged == 1) {
    stream_launch(sm, level, omega, r32, x, s);
    return;
  }
  const bool bf = sm->prec == RAV_BF16_FACT;
  if (g.dim == 2) {
    if (bf) launch_staged_t<2, __nv_bfloat16, 2>(g, SL, omega, r32, x, s);
    else launch_staged_t<2, float, 2>(g, SL, omega, r32, x, s);
  } else {
    if (SL.staged == 2) {
      if (bf) launch_staged_t<3, __nv_bfloat16, 2>(g, SL, omega, r32, x, s);
      else launch_staged_t<3, float, 2>(g, SL, omega, r32, x, s);
    } else {
      if (bf) launch_staged_t<3, __nv_bfloat16, 4>(g, SL, omega, r32, x, s);
      else launch_staged_t<3, float, 4>(g, SL, omega, r32, x, s);
    }
  }
}
