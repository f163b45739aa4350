// Node-blocked residual r = b - L x (Eq. 10) on Q2-Q1 levels.
//
// The gradient form of Eq. 7 makes the velocity block A = I_d (x) K: the d
// rows of a velocity node share their velocity columns and values.  One thread
// takes one velocity node: each stored K entry multiplies the d components of
// x at its column node, each pressure column carries the node's d entries of
// B, and the d rows of the node are written together.  The FP64 work is the
// rows' (d FMAs per K entry and per B entry); the stored operator shrinks by
// about 40 % in 2-D and 60 % in 3-D.  Nodes are grouped by their (K, B) entry
// counts into slices of 32 (a new slice at every change of counts, so every
// lane of a slice runs the same trip counts), column-major inside a slice:
//   columns:  slice s, entry k of lane i at cptr[s] + 32 k + i
//             (k < KL: column node; KL <= k < KL + BL: pressure index),
//   values:   K entry k at vptr[s] + 32 k + i, B entry k, component c at
//             vptr[s] + 32 (KL + d k + c) + i.
// Roundoff entries are left out by the rule of the row-wise copy: an entry is
// kept when it is kept in any of the node's rows.  Dirichlet nodes have no
// entries (KL = 0) and get r = 0.  The pressure rows use a sliced-ELL copy of
// their own (the row-wise format and kernel).  The level's K must be the same
// in every component row, entry for entry; the build checks it and gives up
// otherwise (the level then keeps the row-wise residual).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace rav {

__device__ __forceinline__ double blk_row_threshold(const int64_t* rp, const double* va, int64_t row) {
  double m = 0.0;
  for (int64_t k = rp[row]; k < rp[row + 1]; ++k) m = fmax(m, fabs(va[k]));
  return m * 0x1p-46;
}

// Per velocity node: kept K entries (kcnt) and kept pressure entries (bcnt);
// 0, 0 for Dirichlet nodes.  *bad = 1 if the node's rows differ in pattern or
// in their K values.
template <int D>
__global__ void k_blk_counts(Geo g, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ va, int32_t* __restrict__ kcnt, int32_t* __restrict__ bcnt,
                             int* __restrict__ bad) {
  const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (node >= g.nnode) return;
  const int64_t r0 = D * node;
  const int64_t len = rp[r0 + 1] - rp[r0];
  if (len <= 1) {  // Dirichlet identity rows
    kcnt[node] = 0;
    bcnt[node] = 0;
    return;
  }
  double thr = 1e300;
  for (int c = 0; c < D; ++c) {
    if (rp[r0 + c + 1] - rp[r0 + c] != len) atomicExch(bad, 1);
    thr = fmin(thr, blk_row_threshold(rp, va, r0 + c));
  }
  int nk = 0, nb = 0;
  for (int64_t j = 0; j < len; ++j) {
    const int64_t col0 = ci[rp[r0] + j];
    double m = 0.0;
    for (int c = 0; c < D; ++c) {
      const int64_t k = rp[r0 + c] + j;
      m = fmax(m, fabs(va[k]));
      if (col0 < g.n_u) {
        if (ci[k] != col0 + c || va[k] != va[rp[r0] + j]) atomicExch(bad, 1);
      } else if (ci[k] != col0) {
        atomicExch(bad, 1);
      }
    }
    if (!(m > thr)) continue;
    if (col0 < g.n_u) ++nk;
    else ++nb;
  }
  kcnt[node] = nk;
  bcnt[node] = nb;
}

template <int D>
__global__ void k_blk_fill(Geo g, int64_t nslots, const int32_t* __restrict__ bperm, const int64_t* __restrict__ cptr,
                           const int64_t* __restrict__ vptr, const int32_t* __restrict__ kl,
                           const int32_t* __restrict__ bl, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ va, int32_t* __restrict__ col, double* __restrict__ val) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nslots) return;
  const int64_t s = t >> 5;
  const int lane = (int)(t & 31);
  const int32_t node = bperm[t];
  const int KL = kl[s], BL = bl[s];
  int32_t* cp = col + cptr[s] + lane;
  double* vp = val + vptr[s] + lane;
  if (node < 0) {  // padding slot: zero entries on column 0 / pressure 0
    for (int k = 0; k < KL + BL; ++k) cp[32 * k] = 0;
    for (int k = 0; k < KL + D * BL; ++k) vp[32 * k] = 0.0;
    return;
  }
  if (KL == 0) return;
  const int64_t r0 = D * (int64_t)node;
  const int64_t len = rp[r0 + 1] - rp[r0];
  double thr = 1e300;
  for (int c = 0; c < D; ++c) thr = fmin(thr, blk_row_threshold(rp, va, r0 + c));
  int k = 0, kb = 0;
  for (int64_t j = 0; j < len; ++j) {
    const int64_t col0 = ci[rp[r0] + j];
    double m = 0.0;
    for (int c = 0; c < D; ++c) m = fmax(m, fabs(va[rp[r0 + c] + j]));
    if (!(m > thr)) continue;
    if (col0 < g.n_u) {
      cp[32 * k] = (int32_t)(col0 / D);
      vp[32 * k] = va[rp[r0] + j];
      ++k;
    } else {
      cp[32 * (KL + kb)] = (int32_t)(col0 - g.n_u);
      for (int c = 0; c < D; ++c) vp[32 * (KL + D * kb + c)] = va[rp[r0 + c] + j];
      ++kb;
    }
  }
}

// Pressure slices: slot t copies the entries of the row held by slot src[t]
// of the row-wise copy (zeros for padding slots).
__global__ void k_pslice_fill(int64_t nslots, const int64_t* __restrict__ src, const int64_t* __restrict__ pptr,
                              const int32_t* __restrict__ plen, const int64_t* __restrict__ sptr,
                              const int32_t* __restrict__ scol, const double* __restrict__ sval,
                              int32_t* __restrict__ pcol, double* __restrict__ pval) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nslots) return;
  const int64_t ps = t >> 5;
  const int lane = (int)(t & 31);
  const int len = plen[ps];
  const int64_t st = src[t];
  for (int k = 0; k < len; ++k) {
    const int64_t o = pptr[ps] + 32 * (int64_t)k + lane;
    if (st < 0) {
      pcol[o] = 0;
      pval[o] = 0.0;
    } else {
      const int64_t so = sptr[st >> 5] + 32 * (int64_t)k + (st & 31);
      pcol[o] = scol[so];
      pval[o] = sval[so];
    }
  }
}

// r = b - L x on the velocity rows, one thread per node (see above), with the
// same outputs as k_residual_sell (r, optional fp32 copy, per-block partial
// sums of r^2).
template <int D>
__global__ void __launch_bounds__(256) k_residual_blk(int64_t nslots, int64_t n_u, const int32_t* __restrict__ bperm,
                                                      const int64_t* __restrict__ cptr,
                                                      const int64_t* __restrict__ vptr,
                                                      const int32_t* __restrict__ kl, const int32_t* __restrict__ bl,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ val, const double* __restrict__ x,
                                                      const double* __restrict__ b, double* __restrict__ r,
                                                      double* __restrict__ part, float* __restrict__ r32) {
  double acc2 = 0.0;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < nslots) {
    const int64_t s = t >> 5;
    const int lane = (int)(t & 31);
    const int32_t node = bperm[t];
    const int KL = kl[s], BL = bl[s];
    double acc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) acc[c] = 0.0;
    if (KL > 0) {
      const int32_t* cp = col + cptr[s] + lane;
      const double* vp = val + vptr[s] + lane;
      int k = 0;
      for (; k + 4 <= KL; k += 4) {  // four column nodes in flight
        int jk[4];
        double vk[4], xk[4][D];
#pragma unroll
        for (int q = 0; q < 4; ++q) jk[q] = ld_stream(cp + 32 * (k + q));
#pragma unroll
        for (int q = 0; q < 4; ++q) vk[q] = ld_stream(vp + 32 * (k + q));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if constexpr (D == 2) {
            const double2 xv = *reinterpret_cast<const double2*>(x + 2 * (int64_t)jk[q]);
            xk[q][0] = xv.x;
            xk[q][1] = xv.y;
          } else {
#pragma unroll
            for (int c = 0; c < D; ++c) xk[q][c] = x[D * (int64_t)jk[q] + c];
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int c = 0; c < D; ++c) acc[c] += vk[q] * xk[q][c];
      }
      for (; k < KL; ++k) {
        const int64_t j = ld_stream(cp + 32 * k);
        const double v = ld_stream(vp + 32 * k);
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] += v * x[D * j + c];
      }
      for (int kb = 0; kb < BL; ++kb) {
        const double xp = x[n_u + ld_stream(cp + 32 * (KL + kb))];
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] += ld_stream(vp + 32 * (KL + D * kb + c)) * xp;
      }
    }
    if (node >= 0) {
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const int64_t row = D * (int64_t)node + c;
        const double rv = KL > 0 ? b[row] - acc[c] : 0.0;
        r[row] = rv;
        if (r32) r32[row] = (float)rv;
        acc2 += rv * rv;
      }
    }
  }
  if (part) {
    const double bs = block_sum(acc2);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
  }
}

}  // namespace rav

namespace rav {

void blocked_free(Level& L) {
  for (void* p : {(void*)L.bperm, (void*)L.bcptr, (void*)L.bvptr, (void*)L.bkl, (void*)L.bbl, (void*)L.bcol,
                  (void*)L.bval, (void*)L.psperm, (void*)L.psptr, (void*)L.pslen, (void*)L.pscol, (void*)L.psval})
    cudaFree(p);
  L.bperm = nullptr;
  L.bcptr = L.bvptr = nullptr;
  L.bkl = L.bbl = L.bcol = nullptr;
  L.bval = nullptr;
  L.psperm = nullptr;
  L.psptr = nullptr;
  L.pslen = L.pscol = nullptr;
  L.psval = nullptr;
  L.nbslice = L.npslice = 0;
  L.rblock = false;
}

// Builds the node-blocked velocity copy and the pressure-row sliced-ELL copy
// of level L (Q2-Q1).  RAV_OK with L.nbslice == 0 when the level's component
// rows do not share K (nothing is kept then).
int blocked_build(Level& L, cudaStream_t s) {
  const Geo& g = L.g;
  if (g.q != 2 || L.nbslice) return RAV_OK;
  const int64_t nn = g.nnode;
  int32_t *kc = nullptr, *bc = nullptr;
  int* bad = nullptr;
  RAV_CUDA(cudaMallocAsync(&kc, sizeof(int32_t) * nn, s));
  RAV_CUDA(cudaMallocAsync(&bc, sizeof(int32_t) * nn, s));
  RAV_CUDA(cudaMallocAsync(&bad, sizeof(int), s));
  RAV_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  const unsigned gb = (unsigned)((nn + 255) / 256);
  if (g.dim == 2) k_blk_counts<2><<<gb, 256, 0, s>>>(g, L.rp, L.ci, L.va, kc, bc, bad);
  else k_blk_counts<3><<<gb, 256, 0, s>>>(g, L.rp, L.ci, L.va, kc, bc, bad);
  std::vector<int32_t> hk(nn), hb(nn);
  int hbad = 0;
  RAV_CUDA(cudaMemcpyAsync(hk.data(), kc, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, s));
  RAV_CUDA(cudaMemcpyAsync(hb.data(), bc, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, s));
  RAV_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  RAV_CUDA(cudaStreamSynchronize(s));
  cudaFreeAsync(kc, s);
  cudaFreeAsync(bc, s);
  cudaFreeAsync(bad, s);
  if (hbad) return RAV_OK;
  // slices of 32 nodes of equal (KL, BL), most entries first
  std::vector<int64_t> order(nn);
  for (int64_t i = 0; i < nn; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return hk[a] != hk[b] ? hk[a] > hk[b] : hb[a] > hb[b];
  });
  std::vector<int32_t> perm, kl, bl;
  std::vector<int64_t> cptr(1, 0), vptr(1, 0);
  for (int64_t i = 0; i < nn;) {
    int64_t j = i;
    while (j < nn && j - i < 32 && hk[order[j]] == hk[order[i]] && hb[order[j]] == hb[order[i]]) ++j;
    for (int64_t q = 0; q < 32; ++q) perm.push_back(i + q < j ? (int32_t)order[i + q] : -1);
    kl.push_back(hk[order[i]]);
    bl.push_back(hb[order[i]]);
    cptr.push_back(cptr.back() + 32 * (int64_t)(hk[order[i]] + hb[order[i]]));
    vptr.push_back(vptr.back() + 32 * (int64_t)(hk[order[i]] + g.dim * hb[order[i]]));
    i = j;
  }
  L.nbslice = (int64_t)kl.size();
  RAV_CUDA(cudaMalloc(&L.bperm, sizeof(int32_t) * perm.size()));
  RAV_CUDA(cudaMalloc(&L.bcptr, sizeof(int64_t) * cptr.size()));
  RAV_CUDA(cudaMalloc(&L.bvptr, sizeof(int64_t) * vptr.size()));
  RAV_CUDA(cudaMalloc(&L.bkl, sizeof(int32_t) * kl.size()));
  RAV_CUDA(cudaMalloc(&L.bbl, sizeof(int32_t) * bl.size()));
  RAV_CUDA(cudaMalloc(&L.bcol, sizeof(int32_t) * std::max<int64_t>(cptr.back(), 1)));
  RAV_CUDA(cudaMalloc(&L.bval, sizeof(double) * std::max<int64_t>(vptr.back(), 1)));
  RAV_CUDA(cudaMemcpy(L.bperm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice));
  RAV_CUDA(cudaMemcpy(L.bcptr, cptr.data(), sizeof(int64_t) * cptr.size(), cudaMemcpyHostToDevice));
  RAV_CUDA(cudaMemcpy(L.bvptr, vptr.data(), sizeof(int64_t) * vptr.size(), cudaMemcpyHostToDevice));
  RAV_CUDA(cudaMemcpy(L.bkl, kl.data(), sizeof(int32_t) * kl.size(), cudaMemcpyHostToDevice));
  RAV_CUDA(cudaMemcpy(L.bbl, bl.data(), sizeof(int32_t) * bl.size(), cudaMemcpyHostToDevice));
  const int64_t nslots = L.nbslice * 32;
  if (g.dim == 2)
    k_blk_fill<2><<<(unsigned)((nslots + 255) / 256), 256, 0, s>>>(g, nslots, L.bperm, L.bcptr, L.bvptr, L.bkl, L.bbl,
                                                                   L.rp, L.ci, L.va, L.bcol, L.bval);
  else
    k_blk_fill<3><<<(unsigned)((nslots + 255) / 256), 256, 0, s>>>(g, nslots, L.bperm, L.bcptr, L.bvptr, L.bkl, L.bbl,
                                                                   L.rp, L.ci, L.va, L.bcol, L.bval);
  RAV_CUDA(cudaGetLastError());
  // the pressure rows: their slots of the row-wise copy, gathered slice by slice
  std::vector<int32_t> sperm(L.nslice * 32), slen(L.nslice);
  std::vector<int64_t> sptr(L.nslice + 1);
  RAV_CUDA(cudaMemcpyAsync(sperm.data(), L.sperm, sizeof(int32_t) * sperm.size(), cudaMemcpyDeviceToHost, s));
  RAV_CUDA(cudaMemcpyAsync(slen.data(), L.slen, sizeof(int32_t) * slen.size(), cudaMemcpyDeviceToHost, s));
  RAV_CUDA(cudaMemcpyAsync(sptr.data(), L.sptr, sizeof(int64_t) * sptr.size(), cudaMemcpyDeviceToHost, s));
  RAV_CUDA(cudaStreamSynchronize(s));
  // pressure rows grouped by their length in the row-wise copy, 32 per slice
  std::vector<std::pair<int32_t, int32_t>> prow;  // (length, row)
  std::vector<int64_t> src_of_row(g.n, -1);       // slot of each row in the row-wise copy
  for (int64_t t = 0; t < (int64_t)sperm.size(); ++t)
    if (sperm[t] >= 0) src_of_row[sperm[t]] = t;
  for (int64_t row = g.n_u; row < g.n; ++row) prow.push_back({slen[src_of_row[row] >> 5], (int32_t)row});
  std::stable_sort(prow.begin(), prow.end(), [](const std::pair<int32_t, int32_t>& a,
                                                const std::pair<int32_t, int32_t>& b) { return a.first > b.first; });
  std::vector<int32_t> pperm, plen;
  std::vector<int64_t> pptr(1, 0);
  for (size_t i = 0; i < prow.size();) {
    size_t j = i;
    while (j < prow.size() && j - i < 32 && prow[j].first == prow[i].first) ++j;
    for (size_t q = 0; q < 32; ++q) pperm.push_back(i + q < j ? prow[i + q].second : -1);
    plen.push_back(prow[i].first);
    pptr.push_back(pptr.back() + 32 * (int64_t)prow[i].first);
    i = j;
  }
  L.npslice = (int64_t)plen.size();
  std::vector<int64_t> psrc(pperm.size(), -1);  // slot of each pressure slot's row in the row-wise copy
  for (size_t t = 0; t < pperm.size(); ++t)
    if (pperm[t] >= 0) psrc[t] = src_of_row[pperm[t]];
  int64_t* psrc_d = nullptr;
  RAV_CUDA(cudaMalloc(&L.psperm, sizeof(int32_t) * pperm.size()));
  RAV_CUDA(cudaMalloc(&L.psptr, sizeof(int64_t) * pptr.size()));
  RAV_CUDA(cudaMalloc(&L.pslen, sizeof(int32_t) * plen.size()));
  RAV_CUDA(cudaMalloc(&L.pscol, sizeof(int32_t) * std::max<int64_t>(pptr.back(), 1)));
  RAV_CUDA(cudaMalloc(&L.psval, sizeof(double) * std::max<int64_t>(pptr.back(), 1)));
  RAV_CUDA(cudaMallocAsync(&psrc_d, sizeof(int64_t) * psrc.size(), s));
  RAV_CUDA(cudaMemcpy(L.psperm, pperm.data(), sizeof(int32_t) * pperm.size(), cudaMemcpyHostToDevice));
  RAV_CUDA(cudaMemcpy(L.psptr, pptr.data(), sizeof(int64_t) * pptr.size(), cudaMemcpyHostToDevice));
  RAV_CUDA(cudaMemcpy(L.pslen, plen.data(), sizeof(int32_t) * plen.size(), cudaMemcpyHostToDevice));
  RAV_CUDA(cudaMemcpyAsync(psrc_d, psrc.data(), sizeof(int64_t) * psrc.size(), cudaMemcpyHostToDevice, s));
  const int64_t nps = L.npslice * 32;
  k_pslice_fill<<<(unsigned)((nps + 255) / 256), 256, 0, s>>>(nps, psrc_d, L.psptr, L.pslen, L.sptr, L.scol, L.sval,
                                                             L.pscol, L.psval);
  RAV_CUDA(cudaGetLastError());
  cudaFreeAsync(psrc_d, s);
  RAV_CUDA(cudaStreamSynchronize(s));
  return RAV_OK;
}

// Blocks of the two launches of one node-blocked residual (velocity nodes,
// pressure rows) with 256 threads each.
int64_t blocked_blocks(const Level& L) { return L.nbslice * 32 / 256 + 1 + (L.npslice * 32 + 255) / 256; }

// One node-blocked residual of level L; part (optional) receives
// blocked_blocks(L) partial sums.
void blocked_launch(const Level& L, const double* x, const double* b, double* r, double* part, float* r32,
                    cudaStream_t s) {
  const int64_t nv = L.nbslice * 32, np = L.npslice * 32;
  const int64_t bv = nv / 256 + 1, bp = (np + 255) / 256;
  if (L.g.dim == 2)
    k_residual_blk<2><<<(unsigned)bv, 256, 0, s>>>(nv, L.g.n_u, L.bperm, L.bcptr, L.bvptr, L.bkl, L.bbl, L.bcol,
                                                   L.bval, x, b, r, part, r32);
  else
    k_residual_blk<3><<<(unsigned)bv, 256, 0, s>>>(nv, L.g.n_u, L.bperm, L.bcptr, L.bvptr, L.bkl, L.bbl, L.bcol,
                                                   L.bval, x, b, r, part, r32);
  if (bp) launch_residual_rows(np, L.psperm, L.psptr, L.pslen, L.pscol, L.psval, x, b, r, part ? part + bv : nullptr,
                               r32, s);
}

}  // namespace rav
