// Streamed subdomain apply, one thread per subdomain, for the reduced
// factored storage (RAV_F32_FACT, RAV_BF16_FACT) on Q2-Q1 levels.
//
// Same arithmetic as k_rav_apply_fact and k_rav_apply_staged (Eq. 13 through
// the block form of L_i^{-1}, A_i = I_d (x) K_i, one pressure DoF):
//   tau = (1/s) (w^T r_u - r_p),
//   y(m,c) = sum_n K^{-1}[m,n] r(n,c) + w(m,c) tau   for the owned nodes m,
//   y_p = -tau,   x[owned] += omega_i y,
// products accumulated in fp32 from the fp32-rounded residual, box nodes n in
// order.  What differs is the layout, chosen so that a thread spends its
// instructions on the FMAs:
//
// * Tiles of compile-time shape.  A block takes a tile of TX x (TY P) (x TZ)
//   vertices, one thread per vertex of a TX x TY (x TZ) slab and P slabs in
//   turn (2-D: 16 x 8 threads, P = 3; 3-D: one warp, 3 x 3 x 3), so that the
//   tiles of a 512^2 or 32^3 level are resident at once (one wave).  The box
//   nodes 2 v0 - 2 .. 2 (v0 + T) of the whole tile are copied once from the
//   fp32 residual into shared memory (zero outside the domain; r is zero on
//   Dirichlet rows already), so box node a of a subdomain is a shared-memory
//   load at a compile-time offset from the thread's corner.
// * One thread per subdomain: no partial sums to combine, the owned rows'
//   accumulators stay in registers (pairs of rows for the packed fp32 FMA)
//   and the w values of the owned nodes are kept when their box node passes.
// * Streaming.  The chunks of a warp (per box node: the 2^d values
//   K^{-1}[q, n] and, in a second array, the d values w(n, c), zero padded to
//   WC) are contiguous: chunk ((b W + warp) NJT + J) 32 + lane, step J = p NV +
//   n of slab p.  Every thread keeps kSmRing steps in flight in registers
//   (evict-first loads; slot u mod kSmRing of the 25 nodes of a box plane,
//   known at compile time), the load of step J + kSmRing issued as step J is
//   consumed; the ring runs on from one plane or slab into the next.  Threads
//   without a subdomain (tiles past the grid's last vertex) load nothing.
// * Restricted scatter: plain fp64 read-modify-writes of the owned DoFs of x,
//   disjoint between subdomains, no atomics.
// The chunks are rebuilt from the grouped factored storage (k_restream), so
// they hold exactly the same rounded values.
#include <cuda_bf16.h>

#include <cmath>

#include "box.cuh"
#include "common.cuh"
#include "cpasync.cuh"
#include "fmt.cuh"

namespace rav {

template <int D>
struct StreamTile;
template <>
struct StreamTile<2> {
  static constexpr int TX = 16, TY = 8, TZ = 1, P = 3, W = 4;
};
template <>
struct StreamTile<3> {
  static constexpr int TX = 3, TY = 3, TZ = 3, P = 1, W = 1;
};

constexpr int kSmRing = 5;  // node steps in flight per thread (divides the 25 nodes of a plane)

template <int D, typename T>
struct StreamPlan {
  using ST = StreamTile<D>;
  static constexpr int NV = BoxT<D>::NV, NON = BoxT<D>::NON;
  static constexpr int WC = D == 3 ? 4 : 2;  // w values per chunk (3-D: 3 and a zero)
  static constexpr int CK = NON * (int)sizeof(T), CW = WC * (int)sizeof(T);
  static constexpr int NT = ST::W * 32;                // threads per block
  static constexpr int TS = ST::TX * ST::TY * ST::TZ;  // subdomains per slab
  static constexpr int NJT = ST::P * NV;               // node steps per thread
  static constexpr int SX = 2 * ST::TX + 3, SY = 2 * ST::TY * ST::P + 3, SZ = D == 3 ? 2 * ST::TZ + 3 : 1;
  static constexpr int RS = D == 3 ? 16 : 8;  // bytes per staged node
  static constexpr size_t BYTES = ((size_t)SX * SY * SZ * RS + 15) / 16 * 16;
  static_assert(TS <= NT, "one thread per subdomain of a slab");
  static_assert(25 % kSmRing == 0 && kSmRing <= NV, "ring slots repeat with every plane of 25 box nodes");
};

template <int D, typename T>
__global__ void __launch_bounds__(StreamTile<D>::W * 32, D == 2 ? 5 : 10)
    k_rav_apply_stream(Geo g, int nbx, int nby, const T* __restrict__ kq, const T* __restrict__ wq,
                       const float* __restrict__ sinv, const double* __restrict__ omega,
                       const float* __restrict__ r32, double* __restrict__ x) {
  using ST = StreamTile<D>;
  using P = StreamPlan<D, T>;
  using RV = typename NodeT<D>::type;
  constexpr int NV = P::NV, NON = P::NON, WC = P::WC, CK = P::CK, CW = P::CW, NJT = P::NJT;
  constexpr int SX = P::SX, SY = P::SY, SZ = P::SZ, R = kSmRing;
  extern __shared__ __align__(16) uint8_t sraw[];
  RV* tile = reinterpret_cast<RV*>(sraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x;
  const int bx = b % nbx, by = (b / nbx) % nby, bz = D == 3 ? b / (nbx * nby) : 0;
  const int o0 = bx * ST::TX, o1 = by * ST::TY * ST::P, o2 = bz * ST::TZ;  // the tile's first vertex
  const int64_t M = g.M;

  // the tile's residual boxes, one warp per staged row of SX nodes
  // (contiguous in r along axis 0), one copy group
  {
    const int64_t J0s = 2 * (int64_t)o0 - 2;
    for (int row = warp; row < SY * SZ; row += ST::W) {
      const int i1 = row % SY, i2 = row / SY;
      const int64_t J1 = 2 * (int64_t)o1 - 2 + i1, J2 = D == 3 ? 2 * (int64_t)o2 - 2 + i2 : 0;
      const bool rin = J1 >= 0 && J1 < M && J2 >= 0 && J2 < M;
      const int64_t rnode = J0s + M * (J1 + M * J2);  // node of the row's first staged position
      RV* drow = tile + row * SX;
      if constexpr (D == 2) {
        for (int i0 = lane; i0 < SX; i0 += 32) {
          const bool in = rin && J0s + i0 >= 0 && J0s + i0 < M;
          st_copy8z(drow + i0, r32 + (in ? 2 * (rnode + i0) : 0), in);
        }
      } else {  // 3 floats a node, the 4th (padding) is never read
        for (int f = lane; f < 3 * SX; f += 32) {
          const int i0 = f / 3, c = f - 3 * i0;
          const bool in = rin && J0s + i0 >= 0 && J0s + i0 < M;
          st_copy4z(reinterpret_cast<float*>(drow + i0) + c, r32 + (in ? 3 * (rnode + i0) + c : 0), in);
        }
      }
    }
  }
  st_commit();

  // this thread's vertex in slab p: (v0, o1 + p TY + ly, v2)
  const int lt = tid < P::TS ? tid : 0;  // threads without a subdomain read inside the tile
  const int lx = lt % ST::TX, ly = (lt / ST::TX) % ST::TY, lz = D == 3 ? lt / (ST::TX * ST::TY) : 0;
  const int v0 = o0 + lx, v2 = o2 + lz;
  unsigned act = 0;  // bit p: the thread has a subdomain in slab p (a prefix of the slabs)
#pragma unroll
  for (int p = 0; p < ST::P; ++p)
    act |= (unsigned)(tid < P::TS && v0 <= g.N && o1 + p * ST::TY + ly <= g.N && (D == 2 || v2 <= g.N)) << p;
  const size_t c0 = ((size_t)b * ST::W + warp) * NJT * 32 + lane;  // chunk of step 0
  const T* kme = kq + c0 * NON;
  const T* wme = wq + c0 * WC;
  // the first R node steps (slab 0) in flight while the tile lands
  RawChunk<CK> kb[R];
  RawChunk<CW> wb[R];
#pragma unroll
  for (int J = 0; J < R; ++J) {
    if (act & 1u) {
      kb[J] = ld_raw<CK>(kme + (size_t)J * 32 * NON);
      wb[J] = ld_raw<CW>(wme + (size_t)J * 32 * WC);
    } else {
#pragma unroll
      for (int i = 0; i < CK / 4; ++i) kb[J].w[i] = 0u;
#pragma unroll
      for (int i = 0; i < CW / 4; ++i) wb[J].w[i] = 0u;
    }
  }
  st_wait<0>();  // the tile has landed
  __syncthreads();

#pragma unroll 1
  for (int p = 0; p < ST::P; ++p) {
    const bool actp = (act >> p) & 1u;
    const int v1 = o1 + p * ST::TY + ly;
    const int v[3] = {v0, v1, v2};
    const int64_t nb = 2 * (int64_t)v0 + M * (2 * (int64_t)v1 + M * (2 * (int64_t)v2));  // node J = 2 v
    // owned node q (bit d = offset on axis d) is free iff 1 <= 2 v + delta <= 2N - 1 per axis
    bool okl[3] = {true, true, true}, okh[3] = {true, true, true};
#pragma unroll
    for (int d = 0; d < D; ++d) {
      okh[d] = v[d] <= g.N - 1;
      okl[d] = okh[d] && v[d] >= 1;
    }
    auto own_ok = [&](int q) {
      bool ok = true;
#pragma unroll
      for (int d = 0; d < D; ++d) ok = ok && (((q >> d) & 1) ? okh[d] : okl[d]);
      return ok;
    };
    auto own_node = [&](int q) { return nb + (q & 1) + M * (((q >> 1) & 1) + M * (q >> 2)); };
    if (actp) {  // the x values written at the end go to L2 now
#pragma unroll
      for (int q = 0; q < NON; ++q)
        if (own_ok(q)) {
          const double* xq = x + D * own_node(q);
          asm volatile("prefetch.global.L2 [%0];" ::"l"(xq));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(xq + D - 1));
        }
    }
    // y2[h][c] = (y(2h, c), y(2h + 1, c)): owned rows in pairs for the packed
    // fp32 FMA (each lane rounds like fmaf)
    float2 y2[NON / 2][D];
    float wo[NON][D];  // w of the owned nodes, kept as their box nodes pass
    float tw = 0.f;
#pragma unroll
    for (int h = 0; h < NON / 2; ++h)
#pragma unroll
      for (int c = 0; c < D; ++c) y2[h][c] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NON; ++q)
#pragma unroll
      for (int c = 0; c < D; ++c) wo[q][c] = 0.f;
    const int tb = ((D == 3 ? 2 * lz * SY : 0) + 2 * (p * ST::TY + ly)) * SX + 2 * lx;  // box node 0
#pragma unroll 1
    for (int a2 = 0; a2 < (D == 3 ? 5 : 1); ++a2) {
#pragma unroll
      for (int u = 0; u < 25; ++u) {
        const int J = p * NV + a2 * 25 + u;
        const int q = u % R;  // slot of step J (known once the plane is unrolled)
        float kf[NON], wf[WC];
        widen_words<T, CK / 4>(kb[q].w, kf);
        widen_words<T, CW / 4>(wb[q].w, wf);
        const RV rv = tile[tb + (a2 * SY + u / 5) * SX + u % 5];
        float rc[D];
        rc[0] = rv.x;
        rc[1] = rv.y;
        if constexpr (D == 3) rc[2] = reinterpret_cast<const float4&>(rv).z;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const float2 rr = make_float2(rc[c], rc[c]);
#pragma unroll
          for (int h = 0; h < NON / 2; ++h)
            y2[h][c] = __ffma2_rn(make_float2(kf[2 * h], kf[2 * h + 1]), rr, y2[h][c]);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) tw = fmaf(wf[c], rc[c], tw);
        // box node (2 + d0, 2 + d1, 2 + d2) is owned node d0 + 2 d1 + 4 d2
        if (u % 5 >= 2 && u % 5 <= 3 && u / 5 >= 2 && u / 5 <= 3) {
          const int qo = (u % 5 - 2) + 2 * (u / 5 - 2);
          if constexpr (D == 2) {
#pragma unroll
            for (int c = 0; c < D; ++c) wo[qo][c] = wf[c];
          } else {  // plane a2 = 2 + d2
#pragma unroll
            for (int c = 0; c < D; ++c) {
              wo[qo][c] = a2 == 2 ? wf[c] : wo[qo][c];
              wo[qo + 4][c] = a2 == 3 ? wf[c] : wo[qo + 4][c];
            }
          }
        }
        // the slot is read (its values are in the FMAs above): refill it with step J + R
        const int Jn = J + R;
        const bool an = (act >> (Jn < (p + 1) * NV ? p : p + 1)) & 1u;  // slab of step Jn
        if (Jn < NJT && an) {
          kb[q] = ld_raw<CK>(kme + (size_t)Jn * 32 * NON);
          wb[q] = ld_raw<CW>(wme + (size_t)Jn * 32 * WC);
        }
      }
    }
    if (actp) {
      const int64_t pid = v0 + (int64_t)(g.N + 1) * (v1 + (int64_t)(g.N + 1) * v2);
      const float tau = sinv[(((size_t)b * ST::W + warp) * ST::P + p) * 32 + lane] * (tw - r32[g.n_u + pid]);
      const double om = omega[pid];
#pragma unroll
      for (int q = 0; q < NON; ++q) {
        if (!own_ok(q)) continue;
        double* xq = x + D * own_node(q);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const float yv = (q & 1) ? y2[q >> 1][c].y : y2[q >> 1][c].x;
          xq[c] = xq[c] + om * (double)(yv + wo[q][c] * tau);
        }
      }
      x[g.n_u + pid] += om * (double)-tau;
    }
  }
}

// Builds the streamed chunks from the grouped factored storage (K^{-1} rows of
// unit u = p 2^d + q at ((u / G) NV + n) G + u % G, G = 2^lg; w and 1/s per
// subdomain, NV d + 1 values): one thread per (subdomain, box node).  Values
// are copied bit for bit; 1/s is widened to fp32.
template <int D, typename T>
__global__ void k_restream(Geo g, int nbx, int nby, const T* __restrict__ kinv, const T* __restrict__ ws, int lg,
                           T* __restrict__ kq, T* __restrict__ wq, float* __restrict__ sinv) {
  using ST = StreamTile<D>;
  using P = StreamPlan<D, T>;
  constexpr int NV = P::NV, NON = P::NON, WC = P::WC, NWS = D * NV + 1;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= g.n_p * (int64_t)NV) return;
  const int64_t p = e / NV;
  const int n = (int)(e % NV);
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  const int bx = v[0] / ST::TX, lx = v[0] % ST::TX;
  const int by = v[1] / (ST::TY * ST::P), rem = v[1] % (ST::TY * ST::P);
  const int slab = rem / ST::TY, ly = rem % ST::TY;
  const int bz = D == 3 ? v[2] / ST::TZ : 0, lz = D == 3 ? v[2] % ST::TZ : 0;
  const int l = lx + ST::TX * (ly + ST::TY * lz);
  const int warp = l >> 5, lane = l & 31;
  const int64_t b = bx + (int64_t)nbx * (by + (int64_t)nby * bz);
  const int64_t ci = ((b * ST::W + warp) * P::NJT + slab * NV + n) * 32 + lane;
  const int64_t G = int64_t(1) << lg;
#pragma unroll
  for (int q = 0; q < NON; ++q) {
    const int64_t u = p * NON + q;
    kq[ci * NON + q] = kinv[((u >> lg) * NV + n) * G + (u & (G - 1))];
  }
  const T zero = Fmt<T>::enc(0.0);
#pragma unroll
  for (int c = 0; c < WC; ++c) wq[ci * WC + c] = c < D ? ws[p * NWS + n * D + c] : zero;
  if (n == 0)
    sinv[((b * ST::W + warp) * ST::P + slab) * 32 + lane] = Fmt<T>::dec(ws[p * NWS + NWS - 1], nullptr);
}

}  // namespace rav

using namespace rav;

template <int D, typename T>
static int restream_t(const Geo& g, SmLevel& SL, cudaStream_t s) {
  using ST = StreamTile<D>;
  using P = StreamPlan<D, T>;
  const int nv = g.N + 1;
  const int nbx = (nv + ST::TX - 1) / ST::TX;
  const int nby = (nv + ST::TY * ST::P - 1) / (ST::TY * ST::P);
  const int nbz = D == 3 ? (nv + ST::TZ - 1) / ST::TZ : 1;
  const int64_t blocks = (int64_t)nbx * nby * nbz;
  const int64_t chunks = blocks * ST::W * P::NJT * 32;
  staged_free(SL);
  RAV_CUDA(cudaMalloc(&SL.skq, sizeof(T) * chunks * P::NON));
  RAV_CUDA(cudaMalloc(&SL.swq, sizeof(T) * chunks * P::WC));
  RAV_CUDA(cudaMalloc(&SL.ssinv, sizeof(float) * blocks * ST::W * ST::P * 32));
  RAV_CUDA(cudaMemsetAsync(SL.skq, 0, sizeof(T) * chunks * P::NON, s));
  RAV_CUDA(cudaMemsetAsync(SL.swq, 0, sizeof(T) * chunks * P::WC, s));
  RAV_CUDA(cudaMemsetAsync(SL.ssinv, 0, sizeof(float) * blocks * ST::W * ST::P * 32, s));
  int lg = 0;
  while ((1 << lg) < 32 / SL.split) ++lg;
  const int64_t tot = g.n_p * (int64_t)P::NV;
  k_restream<D, T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g, nbx, nby, (const T*)SL.inv, (const T*)SL.ws, lg,
                                                                 (T*)SL.skq, (T*)SL.swq, SL.ssinv);
  RAV_CUDA(cudaGetLastError());
  RAV_CUDA(cudaFuncSetAttribute(k_rav_apply_stream<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)P::BYTES));
  SL.sgeo = StagedGeo{ST::TX, ST::TY * ST::P, ST::TZ, nbx, nby, nbz, ST::W, P::SX, P::SY, P::SZ};
  SL.staged = 1;
  return RAV_OK;
}

// (Re)builds the streamed chunks of a reduced factored Q2-Q1 level (one thread
// per subdomain).
int stream_build(rav_smoother* sm, int level, cudaStream_t s) {
  SmLevel& SL = sm->lev[level];
  const Geo& g = sm->mg->lev[level].g;
  const bool bf = sm->prec == RAV_BF16_FACT;
  if (g.dim == 2) return bf ? restream_t<2, __nv_bfloat16>(g, SL, s) : restream_t<2, float>(g, SL, s);
  return bf ? restream_t<3, __nv_bfloat16>(g, SL, s) : restream_t<3, float>(g, SL, s);
}

template <int D, typename T>
static void launch_stream_t(const Geo& g, const SmLevel& SL, const double* omega, const float* r32, double* x,
                            cudaStream_t s) {
  const StagedGeo& sg = SL.sgeo;
  const unsigned blocks = (unsigned)((int64_t)sg.ntx * sg.nty * sg.ntz);
  k_rav_apply_stream<D, T><<<blocks, StreamTile<D>::W * 32, StreamPlan<D, T>::BYTES, s>>>(
      g, sg.ntx, sg.nty, (const T*)SL.skq, (const T*)SL.swq, SL.ssinv, omega, r32, x);
}

// One streamed apply x += S_RAV r on a level whose chunks are built.
void stream_launch(const rav_smoother* sm, int level, const double* omega, const float* r32, double* x,
                   cudaStream_t s) {
  const SmLevel& SL = sm->lev[level];
  const Geo& g = sm->mg->lev[level].g;
  const bool bf = sm->prec == RAV_BF16_FACT;
  if (g.dim == 2) {
    if (bf) launch_stream_t<2, __nv_bfloat16>(g, SL, omega, r32, x, s);
    else launch_stream_t<2, float>(g, SL, omega, r32, x, s);
  } else {
    if (bf) launch_stream_t<3, __nv_bfloat16>(g, SL, omega, r32, x, s);
    else launch_stream_t<3, float>(g, SL, omega, r32, x, s);
  }
}
