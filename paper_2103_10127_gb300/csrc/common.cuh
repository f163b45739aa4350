// Internal declarations shared by the translation units of libravanka.
// Q2-Q1 Stokes on tensor box grids; numbering and conventions as in ravanka.h.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include "../../include/ravanka.h"

#define RAV_TRY(call)                           \
  do {                                          \
    int rc_ = (call);                           \
    if (rc_ != RAV_OK) return rc_;              \
  } while (0)

#define RAV_CUDA(call)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) {                    \
      rav::note_cuda_error(e_);                 \
      return RAV_ERR_CUDA;                      \
    }                                           \
  } while (0)

namespace rav {

void note_cuda_error(cudaError_t e);
inline cudaStream_t S(rav_stream s) { return reinterpret_cast<cudaStream_t>(s); }

constexpr int kMaxLevels = 16;

// Geometry of one level, passed by value to kernels.
struct Geo {
  int dim;
  int N;
  int q;          // velocity degree: 2 (Q2-Q1) or 1 (stabilised Q1-Q1, velocity nodes = vertices)
  int64_t M;      // velocity nodes per axis, q N + 1
  int64_t nnode;  // M^dim
  int64_t n_u, n_p, n;
  const double* xv[3];  // device vertex coordinates per axis (N + 1)
};

// Per-axis interpolation tables from level l-1 into level l, nonzero weights
// only.  Prolongation: fine Q2 node index I takes pc2[I] coarse nodes
// pk2[3I+j] with weights pw2[3I+j]; fine vertex v takes pc1[v] coarse vertices
// (pk1, pw1, stride 2).  Restriction (the transpose): coarse Q2 node K gathers
// rc2[K] fine nodes rk2[7K+j] with weights rw2[7K+j], fine boundary nodes left
// out (up to 7 per axis on graded grids); coarse vertex K gathers rc1[K] fine
// vertices (rk1, rw1, stride 3).
template <typename W>
struct XferTabT {
  const int* pc2[3];
  const int* pk2[3];
  const W* pw2[3];
  const int* pc1[3];
  const int* pk1[3];
  const W* pw1[3];
  const int* rc2[3];
  const int* rk2[3];
  const W* rw2[3];
  const int* rc1[3];
  const int* rk1[3];
  const W* rw1[3];
};
using XferTab = XferTabT<double>;

struct Level {
  Geo g;
  double* xv_dev[3] = {nullptr, nullptr, nullptr};
  std::vector<double> xv_host[3];
  int64_t nnz = 0;
  int64_t* rp = nullptr;   // CSR row pointer (n + 1)
  int32_t* ci = nullptr;   // CSR columns, ascending per row
  double* va = nullptr;    // CSR values
  // sliced-ELL copy of the operator for the residual: slices of 32 rows of one
  // common length (rows grouped by length), column-major inside a slice
  int64_t nslice = 0;
  int rsplit = 1;  // threads per row of the residual kernel (more on small levels: shorter latency chains)
  int32_t* sperm = nullptr;  // row of slot t = 32 s + lane, -1 for padding
  int32_t* sslot = nullptr;  // slot of row i (the inverse of sperm), for the fused smoothing step
  int64_t* sptr = nullptr;   // offset of slice s in sval/scol
  int32_t* slen = nullptr;   // row length of slice s (1 = Dirichlet identity rows)
  int32_t* scol = nullptr;
  double* sval = nullptr;
  // fp32 residual on levels between the coarsest and the finest
  // (rav_set_coarse_residual_f32): sval rounded to fp32 in the same slots, and
  // a work copy of x in fp32
  float* sval32 = nullptr;
  float* x32 = nullptr;
  // node-blocked residual (blocked.cu, Q2-Q1): velocity nodes in slices of 32
  // by (K, B) entry counts, pressure rows in a sliced-ELL copy of their own;
  // rblock: the residual uses it (chosen per level at set-up)
  bool rblock = false;
  int64_t nbslice = 0, npslice = 0;
  int32_t* bperm = nullptr;
  int64_t* bcptr = nullptr;
  int64_t* bvptr = nullptr;
  int32_t* bkl = nullptr;
  int32_t* bbl = nullptr;
  int32_t* bcol = nullptr;
  double* bval = nullptr;
  int32_t* psperm = nullptr;
  int64_t* psptr = nullptr;
  int32_t* pslen = nullptr;
  int32_t* pscol = nullptr;
  double* psval = nullptr;
  double* x = nullptr;     // level work vectors (coarse levels' iterate and rhs)
  double* b = nullptr;
  double* r = nullptr;     // residual
  // interpolation tables into this level (unused on level 0); one device
  // allocation per axis holding the twelve arrays of XferTab
  void* xfer[3] = {nullptr, nullptr, nullptr};
  XferTab tabs{};
  XferTab tab() const { return tabs; }
  // fp32 transfers (rav_set_transfers_f32): the weights of tabs in fp32 (one
  // allocation per axis, the index arrays shared with tabs), the fp32 residual
  // restricted from this level and the fp32 copy of the coarser level's x
  // prolongated into it
  void* xfer32[3] = {nullptr, nullptr, nullptr};
  XferTabT<float> tabs32{};
  float* rf32 = nullptr;
  float* xc32 = nullptr;
};

}  // namespace rav

struct rav_mg {
  int dim = 2, N = 0, nlev = 0;
  int device = 0;  // CUDA device current at mg_setup (the hierarchy's memory lives there)
  double eta0 = 1.0;
  int bc = 0;
  int elem = RAV_ELEM_Q2Q1;  // discretisation (rav_element)
  double beta = 0.0;         // stabilisation constant of Eq. 8 (Q1-Q1)
  std::vector<double> blobs;   // host copy
  double* blobs_dev = nullptr;
  int nblobs = 0;
  rav::Level lev[rav::kMaxLevels];
  double* cinv = nullptr;      // (n0 + 1)^2 row-major inverse of the bordered coarse system
  double* norm_part = nullptr; // partial sums for norms and dot products
  double* scalar_dev = nullptr;
  double* scalar_host = nullptr;  // pinned, 128 entries
  int part_cap = 0;
  // timing hook (rav_profile_*): event pairs around the solve-path kernels
  unsigned prof_mask = 0;  // bit k: record kernel class k (rav::PROF_*)
  int prof_level = -1;     // record this level only, -1 = all
  struct ProfRec {
    int level, kind;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> ev_free;
  std::vector<ProfRec> ev_used;
  double prof_ms[rav::kMaxLevels][5] = {};
  int64_t prof_cnt[rav::kMaxLevels][5] = {};
  // captured V-cycles, replayed with cudaGraphLaunch (see vcycle in cycle.cu)
  bool use_graphs = true;
  bool coarse_f32 = false;  // fp32 residuals on the levels between the coarsest and the finest
  bool xfer_f32 = false;    // fp32 restriction and prolongation in the V-cycle (Q2-Q1)
  cudaStream_t cap_stream = nullptr;
  struct GraphEntry {
    const rav_smoother* sm;
    const double* x;
    const double* b;
    int nu1, nu2;
    int entry;
    int64_t launches;  // kernels in one replay
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
};

namespace rav {
enum { PROF_APPLY = 0, PROF_RESIDUAL = 1, PROF_RESTRICT = 2, PROF_PROLONG = 3, PROF_COARSE = 4 };
// Start/stop a recorded interval on stream s when class `kind` of `level` is
// being recorded; *start is nullptr otherwise.  Defined in setup.cu.
int prof_begin(rav_mg* mg, int level, int kind, cudaStream_t s, cudaEvent_t* start);
int prof_end(rav_mg* mg, int level, int kind, cudaEvent_t start, cudaStream_t s);
}  // namespace rav

namespace rav {
// Tiling of the staged reduced-precision apply (staged.cu): tiles of
// tx x ty x tz vertices, ntx x nty x ntz of them, wpt warps per tile, staged
// Q2-node block sx x sy x sz (2t + 3 per axis; sz = 1 in 2-D).
struct StagedGeo {
  int tx, ty, tz;
  int ntx, nty, ntz;
  int wpt;
  int sx, sy, sz;
};
}  // namespace rav

// Smoother data of one level: stored inverse rows and damping per subdomain.
struct SmLevel {
  int64_t np = 0, units = 0;
  bool factored = false;     // RAV factored (fp64 / fp32 / bf16): rows of K^{-1} in inv, w and 1/s in ws
  int split = 1;             // factored apply: threads per owned node (storage grouped by 32/split units)
  void* ws = nullptr;
  void* inv = nullptr;       // RAV: packed owned rows; AV/MV: full inverses (fp64, column-major)
  float* scale = nullptr;    // fp8 row scales
  float* r32 = nullptr;      // fp32 residual for reduced-precision storage (n entries)
  double* omega = nullptr;   // damping per subdomain
  double* corr = nullptr;    // AV corrections, n_p x n_box
  // line-search label collection (learn.cu)
  double* lsum = nullptr;    // sum of omega* per subdomain
  int* lcnt = nullptr;       // number of samples
  double* ones = nullptr;    // unit damping
  double* ctmp = nullptr;    // subdomain corrections with unit damping
  double* stmp = nullptr;    // the whole step with the current damping
  double* rtmp = nullptr;    // residual after that step
  double* xalt = nullptr;    // fused smoothing: the second iterate buffer (n entries)
  // staged apply of reduced factored storage (staged.cu, stream.cu): threads
  // per subdomain (0 = not used), tiling and the chunks it streams
  int staged = 0;
  rav::StagedGeo sgeo{};
  void* skq = nullptr;
  void* swq = nullptr;
  float* ssinv = nullptr;
};

struct rav_smoother {
  rav_mg* mg = nullptr;
  int kind = RAV_RAV, prec = RAV_F64;
  double omega = 0.5;
  bool collect = false;  // accumulate line-search labels in each smoothing step
  bool fused = false;    // Q1-Q1 RAV fp64: residual and subdomain apply in one kernel per step
  SmLevel lev[rav::kMaxLevels];
};

// Subdomain apply with an explicit damping array; labels; damping reset
// (smoother.cu, learn.cu).
// r32 (optional): r rounded to fp32; reduced-precision storage reads it (made from r when null).
int apply_with_omega(rav_smoother* sm, int level, const double* r, double* x, const double* omega, cudaStream_t s,
                     const float* r32 = nullptr);
int collect_labels(rav_smoother* sm, int level, const double* r, cudaStream_t s);
// Staged apply (staged.cu): build its chunks for S threads per subdomain (0
// frees them), launch it, release it.
int staged_build(rav_smoother* sm, int level, int S, cudaStream_t s, int cand = 0);
void staged_launch(const rav_smoother* sm, int level, const double* omega, const float* r32, double* x,
                   cudaStream_t s);
void staged_free(SmLevel& SL);
// Streamed apply, one thread per subdomain (stream.cu): the S = 1 case of the above.
int stream_build(rav_smoother* sm, int level, cudaStream_t s);
void stream_launch(const rav_smoother* sm, int level, const double* omega, const float* r32, double* x,
                   cudaStream_t s);
// Node-blocked residual (blocked.cu): build (leaves nbslice 0 where the level
// does not qualify), free, partial-sum blocks of one launch, launch.
namespace rav {
int blocked_build(Level& L, cudaStream_t s);
void blocked_free(Level& L);
int64_t blocked_blocks(const Level& L);
void blocked_launch(const Level& L, const double* x, const double* b, double* r, double* part, float* r32,
                    cudaStream_t s);
// The row-wise residual kernel on a sliced-ELL copy (cycle.cu).
void launch_residual_rows(int64_t nslots, const int32_t* sperm, const int64_t* sptr, const int32_t* slen,
                          const int32_t* scol, const double* sval, const double* x, const double* b, double* r,
                          double* part, float* r32, cudaStream_t s);
}  // namespace rav
int reset_omega(rav_smoother* sm, cudaStream_t s);

namespace rav {
// Process-wide count of the kernels the solve path (residual, subdomain
// apply, transfers, coarse solve, vector updates) has launched.
void note_launch(int k = 1);
}

// ---- device helpers -------------------------------------------------------
namespace rav {

__host__ __device__ inline int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Velocity node tuple of velocity DoF i (i < n_u) and its component.
__device__ inline void vel_node(const Geo& g, int64_t i, int64_t* I, int& c) {
  int64_t id = i / g.dim;
  c = (int)(i - id * g.dim);
  for (int a = 0; a < g.dim; ++a) { I[a] = id % g.M; id /= g.M; }
}
__device__ inline bool node_on_boundary(const Geo& g, const int64_t* I) {
  bool b = false;
  for (int a = 0; a < g.dim; ++a) b |= (I[a] == 0) | (I[a] == g.M - 1);
  return b;
}
__device__ inline bool is_dirichlet(const Geo& g, int64_t i) {
  if (i >= g.n_u) return false;
  int64_t I[3];
  int c;
  vel_node(g, i, I, c);
  return node_on_boundary(g, I);
}
__device__ inline int64_t node_id(const Geo& g, const int64_t* I) {
  int64_t id = 0;
  for (int a = g.dim - 1; a >= 0; --a) id = id * g.M + I[a];
  return id;
}
// Loads of data streamed once per pass (operator values and columns, stored
// inverses) with the evict-first hint, so they do not push the vectors that
// every pass gathers from (x, r) out of L2.
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ __nv_bfloat16 ld_stream(const __nv_bfloat16* p) {
  const unsigned short v = __ldcs(reinterpret_cast<const unsigned short*>(p));
  return __nv_bfloat16(__nv_bfloat16_raw{v});
}

template <int D>
__device__ __forceinline__ int64_t node_id_t(const Geo& g, const int64_t* I) {
  int64_t id = 0;
#pragma unroll
  for (int a = D - 1; a >= 0; --a) id = id * g.M + I[a];
  return id;
}
__device__ inline int64_t vert_id(const Geo& g, const int64_t* v) {
  int64_t id = 0;
  for (int a = g.dim - 1; a >= 0; --a) id = id * (g.N + 1) + v[a];
  return id;
}
__device__ inline double node_coord(const Geo& g, int a, int64_t I) {
  if (g.q == 1) return g.xv[a][I];
  return (I & 1) ? 0.5 * (g.xv[a][(I - 1) >> 1] + g.xv[a][(I + 1) >> 1]) : g.xv[a][I >> 1];
}

// Viscosity eta0 * 10^(max_k s_k exp(-|x - c_k|^2 / (2 rho_k^2))), eta0 without blobs.
struct Coef {
  double eta0;
  int nblobs;
  const double* blobs;  // device, nblobs * 5 (cx, cy, cz, rho, s)
};
__device__ inline double viscosity_at(const Coef& C, int dim, const double* x) {
  if (C.nblobs == 0) return C.eta0;
  double m = 0.0;
  for (int k = 0; k < C.nblobs; ++k) {
    const double* b = C.blobs + 5 * k;
    double d2 = 0.0;
    for (int a = 0; a < dim; ++a) d2 += (x[a] - b[a]) * (x[a] - b[a]);
    const double v = b[4] * exp(-d2 / (2.0 * b[3] * b[3]));
    m = v > m ? v : m;
  }
  return C.eta0 * exp(m * 2.302585092994045684);  // 10^m
}

// Block-wide sum of one double per thread (blockDim.x a multiple of 32, <= 1024).
__device__ inline double block_sum(double v) {
  __shared__ double wsum[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) wsum[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    v = l < nw ? wsum[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

inline int grid_for(int64_t n, int threads, int cap = 152 * 64) {
  int64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// Shared host routines (defined in cycle.cu).
// r32 (optional): the residual rounded to fp32 as well, for applies that accumulate in fp32.
int residual_impl(rav_mg* mg, int level, const double* x, const double* b, double* r, double* norm2_dev,
                  cudaStream_t s, float* r32 = nullptr);
// Threads per coarse DoF of the restriction into the coarse level gc: 8 below
// 2^14 coarse DoF sites, where one thread per site leaves the GPU waiting on
// long fp64 chains, else 1 (the shuffle reduction costs fp64 work of its own);
// the batched restriction uses the same rule.
__host__ __device__ inline int restrict_split(const Geo& gc) {
  return gc.nnode + gc.n_p < (int64_t(1) << 14) ? 8 : 1;
}
int restrict_impl(rav_mg* mg, int level, const double* rf, double* bc, cudaStream_t s);
int prolong_impl(rav_mg* mg, int level, const double* xc, double* xf, cudaStream_t s);
int coarse_impl(rav_mg* mg, const double* b, double* x, cudaStream_t s);
// Deterministic sum of squares / dot product into *out_dev (two kernels).
int dot_impl(rav_mg* mg, const double* a, const double* b, int64_t n, double* out_dev, cudaStream_t s);

}  // namespace rav

// Smoother entry used by the cycle (defined in smoother.cu) and the V-cycle (cycle.cu).
// entry (how x and the level's residual vector stand when smoothing starts):
//   ENTRY_GENERAL  nothing known;
//   ENTRY_X_ZERO   x is 0, so the first residual is b itself (free rows; b is 0
//                  on Dirichlet rows below the finest level): its SpMV is skipped;
//   ENTRY_R_READY  the level's r (and the fp32 copy of reduced storage) already
//                  holds b - L x, computed for a norm: its SpMV is skipped.
// The results are the same in every case.
enum { ENTRY_GENERAL = 0, ENTRY_X_ZERO = 1, ENTRY_R_READY = 2 };
int rav_smooth_impl(rav_smoother* sm, int level, double* x, const double* b, int steps, cudaStream_t s,
                    int entry = ENTRY_GENERAL);
// The fused form of `steps` RAV steps (fused.cu): one kernel per step computes
// the residual on each tile's subdomain boxes and applies the subdomains.
int fused_smooth_impl(rav_smoother* sm, int level, double* x, const double* b, int steps, cudaStream_t s);
namespace rav {
int vcycle_impl(rav_mg* mg, rav_smoother* sm, double* x, const double* b, int nu1, int nu2, int entry,
                cudaStream_t s);
// Destroys the captured V-cycles that use smoother sm (all of them for nullptr).
void drop_graphs(rav_mg* mg, const rav_smoother* sm);
}
