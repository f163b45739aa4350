// Serial FP64 oracle for the restricted additive Vanka (RAV) multigrid method.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
// this file; only the tests, the smoke check and the CPU-baseline leg of the
// benchmark do.  It shares no code with the CUDA library.
//
// What it computes, and where it comes from (Saberi, Meschke, Vogel,
// "A restricted additive Vanka smoother for geometric multigrid"):
//   * Stokes saddle-point system L x = b, L = [A B; B^T C]      (Sec. 2, Eqs. 5-7, 9)
//       A = (eta grad v, grad u), B = -(div v, q); C = 0 for the inf-sup stable
//       Q2-Q1 pair (Sec. 2, remark after Eq. 7), and for the equal-order Q1-Q1
//       pair the pressure stabilisation of Eq. 8,
//       C = -beta sum_e h_e^2 (grad q, grad p)_e, h_e the cell diameter.
//   * Vanka subdomains: pressure DoF p_i plus every velocity DoF of the cells
//     around vertex i (Sec. 3, definition before Eq. 11), taken structurally.
//   * Local systems L_i = R_i L R_i^T and their inverses (Sec. 3, Eq. 11).
//   * Smoothers, each one step of x <- x + S (b - L x) (Eq. 10):
//       multiplicative (Eq. 11, run as the sequential sweep with a residual
//       refresh per subdomain as described around Eq. 15), additive (Eq. 12)
//       and restricted additive (Eq. 13), the latter applying only the owned
//       rows of L_i^{-1} (Sec. 4.3).
//   * Geometric multigrid V-cycle with nu pre = nu post smoothing, LU coarse
//     solve, operators assembled on every level (Sec. 2, Sec. 4 setup).
//   * Stationary iteration to a 1e-8 residual reduction (Sec. 4) and FGMRES(30)
//     with one V-cycle as right preconditioner (Sec. 4, remark on Krylov use).
// Readings where the paper is silent (ownership rule for Q2 edge/face/cell
// nodes, transfer operators, pressure null space, MV order) are stated next to
// the code that implements them.
//
// Plain style on purpose: element loops, sorted CSR with binary search, dense
// LU with partial pivoting.  No blocking, fusion or reordering.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// Threads for the loops over independent subdomains (local inverses and the
// RAV/AV corrections, whose per-subdomain arithmetic does not depend on the
// order); 1 unless orc_set_threads says otherwise.  Every other loop runs
// serially.  Without OpenMP the pragmas are ignored and everything is serial.
int g_threads = 1;

// ---------------------------------------------------------------------------
// 1-D building blocks on the reference interval [0,1].
// Three-point Gauss-Legendre rule (exact to degree 5).
const double kGaussX[3] = {0.5 - 0.3872983346207416885, 0.5, 0.5 + 0.3872983346207416885};
const double kGaussW[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};

// Quadratic Lagrange basis with nodes t = 0, 1/2, 1.
double q2(int a, double t) {
  if (a == 0) return 2.0 * (t - 0.5) * (t - 1.0);
  if (a == 1) return 4.0 * t * (1.0 - t);
  return 2.0 * t * (t - 0.5);
}
double dq2(int a, double t) {
  if (a == 0) return 4.0 * t - 3.0;
  if (a == 1) return 4.0 - 8.0 * t;
  return 4.0 * t - 1.0;
}
// Linear Lagrange basis with nodes t = 0, 1.
double q1(int b, double t) { return b == 0 ? 1.0 - t : t; }

const double kPi = 3.141592653589793238462643383279502884;

// ---------------------------------------------------------------------------
// Problem description (same on every level except the coordinates).
struct Problem {
  int dim = 2;
  double eta0 = 1.0;
  std::vector<double> blobs;  // per blob: cx, cy, cz, rho, s
  int bc = 0;                 // 0 lid-driven cavity, 1 no-slip, 2 quadratic exact solution
  int elem = 0;               // 0 Q2-Q1 (C = 0), 1 stabilised Q1-Q1 (Eq. 8)
  double beta = 0.0;          // stabilisation constant of Eq. 8 (Q1-Q1 only)
};

// Viscosity: eta0 * 10^(max_k s_k exp(-|x-c_k|^2 / (2 rho_k^2))), eta0 when no blobs.
double viscosity(const Problem& P, const double* x) {
  const int nb = (int)P.blobs.size() / 5;
  if (nb == 0) return P.eta0;
  double m = 0.0;
  for (int k = 0; k < nb; ++k) {
    const double* b = &P.blobs[5 * k];
    double d2 = 0.0;
    for (int a = 0; a < P.dim; ++a) d2 += (x[a] - b[a]) * (x[a] - b[a]);
    double v = b[4] * std::exp(-d2 / (2.0 * b[3] * b[3]));
    if (v > m) m = v;
  }
  return P.eta0 * std::exp(m * std::log(10.0));
}

// Body force f(x) for the forcing kinds:
// 0 none; 1 2-D manufactured stream function psi = sin^2(pi x) sin^2(pi y),
//   u = (d psi/dy, -d psi/dx), p = cos(pi x) cos(pi y), f = -eta0 lap u + grad p;
// 2 "sinker" f = (0,..,0,-phi), phi = max_k exp(-|x-c_k|^2/(2 rho_k^2));
// 3 quadratic exact solution u = (y^2, x^2) [3-D: (y^2, z^2, x^2)],
//   p = sum x_a - d/2, f = -eta0 lap u + grad p = (1 - 2 eta0) per component.
void forcing(const Problem& P, int kind, const double* x, double* f) {
  for (int c = 0; c < P.dim; ++c) f[c] = 0.0;
  if (kind == 1) {
    const double X = x[0], Y = x[1], p3 = kPi * kPi * kPi;
    const double lap1 = 2.0 * p3 * std::sin(2 * kPi * Y) * (2.0 * std::cos(2 * kPi * X) - 1.0);
    const double lap2 = -2.0 * p3 * std::sin(2 * kPi * X) * (2.0 * std::cos(2 * kPi * Y) - 1.0);
    f[0] = -P.eta0 * lap1 - kPi * std::sin(kPi * X) * std::cos(kPi * Y);
    f[1] = -P.eta0 * lap2 - kPi * std::cos(kPi * X) * std::sin(kPi * Y);
  } else if (kind == 2) {
    const int nb = (int)P.blobs.size() / 5;
    double m = 0.0;
    for (int k = 0; k < nb; ++k) {
      const double* b = &P.blobs[5 * k];
      double d2 = 0.0;
      for (int a = 0; a < P.dim; ++a) d2 += (x[a] - b[a]) * (x[a] - b[a]);
      double v = std::exp(-d2 / (2.0 * b[3] * b[3]));
      if (v > m) m = v;
    }
    f[P.dim - 1] = -m;
  } else if (kind == 3) {
    for (int c = 0; c < P.dim; ++c) f[c] = 1.0 - 2.0 * P.eta0;
  }
}

// Dirichlet value of velocity component c at boundary point x.
double boundary_value(const Problem& P, const double* x, bool on_top, int c) {
  if (P.bc == 0) return (on_top && c == 0) ? 1.0 : 0.0;  // lid u = e_0, corners included
  if (P.bc == 2) {                                      // quadratic exact solution
    if (P.dim == 2) return c == 0 ? x[1] * x[1] : x[0] * x[0];
    if (c == 0) return x[1] * x[1];
    if (c == 1) return x[2] * x[2];
    return x[0] * x[0];
  }
  return 0.0;
}

// ---------------------------------------------------------------------------
struct Level {
  int dim = 2, N = 0;
  int q = 2;                  // velocity degree: 2 (Q2-Q1) or 1 (Q1-Q1)
  std::vector<double> xv[3];  // vertex coordinates per axis, N+1 each
  int64_t M = 0;              // velocity nodes per axis, q N + 1
  int64_t nnode = 0, n_u = 0, n_p = 0, n = 0;
  std::vector<uint8_t> dir;   // 1 = Dirichlet DoF
  std::vector<double> g;      // Dirichlet values (zero on coarse levels)
  // system matrix, CSR with sorted columns
  std::vector<int64_t> rp;
  std::vector<int64_t> ci;
  std::vector<double> va;
  // prolongation from the next coarser level into this one (rows = this level's DoFs)
  std::vector<int64_t> Prp, Pci;
  std::vector<double> Pva;
  // Vanka data
  std::vector<int64_t> poff, pdof;      // subdomain DoF lists, sorted
  std::vector<int64_t> owner;           // owning subdomain per DoF, -1 for Dirichlet
  std::vector<std::vector<int>> owned;  // local positions of owned DoFs per subdomain
  std::vector<std::vector<double>> inv; // RAV: owned rows of L_i^{-1}; AV/MV: full L_i^{-1}
  std::vector<std::vector<double>> qinv;  // quantised rows (precision emulation)
  std::vector<std::vector<double>> qscale;
  std::vector<double> omega;            // per-subdomain damping
  // coarse bordered LU (coarsest level only)
  std::vector<double> clu;
  std::vector<int64_t> cpiv;
};

struct Oracle {
  Problem P;
  std::vector<Level> lev;  // lev[0] coarsest
  int kind = 0;            // 0 RAV, 1 AV, 2 MV lexicographic, 3 MV coloured
  int prec = 0;            // 0 fp64, 1 fp32, 2 bf16, 3 fp8 e4m3, 5/6 fp32/bf16 factored (RAV only)
  int err = 0;
};

// Index helpers -------------------------------------------------------------
int64_t node_id(const Level& L, const int64_t* I) {
  int64_t id = 0;
  for (int a = L.dim - 1; a >= 0; --a) id = id * L.M + I[a];
  return id;
}
void node_of(const Level& L, int64_t id, int64_t* I) {
  for (int a = 0; a < L.dim; ++a) { I[a] = id % L.M; id /= L.M; }
}
int64_t vert_id(const Level& L, const int64_t* v) {
  int64_t id = 0;
  for (int a = L.dim - 1; a >= 0; --a) id = id * (L.N + 1) + v[a];
  return id;
}
void vert_of(const Level& L, int64_t id, int64_t* v) {
  for (int a = 0; a < L.dim; ++a) { v[a] = id % (L.N + 1); id /= (L.N + 1); }
}
double node_coord(const Level& L, int a, int64_t I) {
  if (L.q == 1) return L.xv[a][I];
  if (I % 2 == 0) return L.xv[a][I / 2];
  return 0.5 * (L.xv[a][(I - 1) / 2] + L.xv[a][(I + 1) / 2]);
}
bool node_on_boundary(const Level& L, const int64_t* I) {
  for (int a = 0; a < L.dim; ++a)
    if (I[a] == 0 || I[a] == L.q * L.N) return true;
  return false;
}

// Cells (per axis) that contain Q2 node index I on an axis with N cells.
int cells_of_node(int64_t I, int N, int64_t* out) {
  int k = 0;
  if (I % 2 == 1) { out[k++] = (I - 1) / 2; return k; }
  if (I / 2 - 1 >= 0) out[k++] = I / 2 - 1;
  if (I / 2 <= N - 1) out[k++] = I / 2;
  return k;
}
// Cells (per axis) that contain vertex index v.
int cells_of_vertex(int64_t v, int N, int64_t* out) {
  int k = 0;
  if (v - 1 >= 0) out[k++] = v - 1;
  if (v <= N - 1) out[k++] = v;
  return k;
}

// Enumerate the tensor product of per-axis lists.
template <class F>
void tensor_loop(int dim, const int* cnt, F&& f) {
  int idx[3] = {0, 0, 0};
  while (true) {
    f(idx);
    int a = 0;
    while (a < dim) {
      if (++idx[a] < cnt[a]) break;
      idx[a] = 0;
      ++a;
    }
    if (a == dim) break;
  }
}

// ---------------------------------------------------------------------------
// Element matrices on cell c (per-axis lower vertex indices).
struct Elem {
  int nl = 9, nv = 4;
  double K[27][27];
  double B[3][27][8];  // B[comp][local velocity node][local Q1 vertex] = -int psi_b d_comp phi_a
  double C[8][8];      // pressure block (Q1-Q1 only)
  double F[27][3];
};

void local_tuple(int dim, int idx, int base, int* t) {
  for (int a = 0; a < dim; ++a) { t[a] = idx % base; idx /= base; }
}

void element(const Oracle& O, const Level& L, const int64_t* c, int fkind, Elem& E) {
  const int d = L.dim;
  E.nl = d == 2 ? 9 : 27;
  E.nv = d == 2 ? 4 : 8;
  std::memset(&E.K, 0, sizeof(E.K));
  std::memset(&E.B, 0, sizeof(E.B));
  std::memset(&E.F, 0, sizeof(E.F));
  double lo[3], h[3];
  for (int a = 0; a < d; ++a) {
    lo[a] = L.xv[a][c[a]];
    h[a] = L.xv[a][c[a] + 1] - lo[a];
  }
  const int nq = E.nl;
  for (int q = 0; q < nq; ++q) {
    int qt[3];
    local_tuple(d, q, 3, qt);
    double xq[3] = {0, 0, 0}, W = 1.0;
    for (int a = 0; a < d; ++a) {
      xq[a] = lo[a] + h[a] * kGaussX[qt[a]];
      W *= kGaussW[qt[a]] * h[a];
    }
    const double eta = viscosity(O.P, xq);
    double fq[3];
    forcing(O.P, fkind, xq, fq);
    double phi[27], grad[27][3], psi[8];
    for (int A = 0; A < E.nl; ++A) {
      int at[3];
      local_tuple(d, A, 3, at);
      double p = 1.0;
      for (int a = 0; a < d; ++a) p *= q2(at[a], kGaussX[qt[a]]);
      phi[A] = p;
      for (int k = 0; k < d; ++k) {
        double gk = dq2(at[k], kGaussX[qt[k]]) / h[k];
        for (int m = 0; m < d; ++m)
          if (m != k) gk *= q2(at[m], kGaussX[qt[m]]);
        grad[A][k] = gk;
      }
    }
    for (int b = 0; b < E.nv; ++b) {
      int bt[3];
      local_tuple(d, b, 2, bt);
      double p = 1.0;
      for (int a = 0; a < d; ++a) p *= q1(bt[a], kGaussX[qt[a]]);
      psi[b] = p;
    }
    for (int A = 0; A < E.nl; ++A) {
      for (int A2 = 0; A2 < E.nl; ++A2) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += grad[A][k] * grad[A2][k];
        E.K[A][A2] += W * eta * s;
      }
      for (int cc = 0; cc < d; ++cc) {
        for (int b = 0; b < E.nv; ++b) E.B[cc][A][b] += -W * psi[b] * grad[A][cc];
        E.F[A][cc] += W * fq[cc] * phi[A];
      }
    }
  }
}

// Element matrices of the stabilised equal-order pair on cell c (Sec. 2, Eq. 7
// with the pressure block of Eq. 8).  Velocity and pressure share the 2^d
// bilinear (trilinear) vertex functions phi_a of the cell:
//   K[a][b]    = int eta grad phi_a . grad phi_b
//   B[c][a][b] = -int phi_b d_c phi_a
//   C[a][b]    = -beta h_e^2 int grad phi_a . grad phi_b, h_e^2 = sum of squared cell sides
//   F[a][c]    = int f_c phi_a
// with the same 3^d-point Gauss rule as the Q2-Q1 element.
void element_q1(const Oracle& O, const Level& L, const int64_t* c, int fkind, Elem& E) {
  const int d = L.dim;
  E.nl = d == 2 ? 4 : 8;
  E.nv = E.nl;
  std::memset(&E.K, 0, sizeof(E.K));
  std::memset(&E.B, 0, sizeof(E.B));
  std::memset(&E.C, 0, sizeof(E.C));
  std::memset(&E.F, 0, sizeof(E.F));
  double lo[3], h[3], diam2 = 0.0;
  for (int a = 0; a < d; ++a) {
    lo[a] = L.xv[a][c[a]];
    h[a] = L.xv[a][c[a] + 1] - lo[a];
    diam2 += h[a] * h[a];
  }
  const int nq = d == 2 ? 9 : 27;
  for (int qp = 0; qp < nq; ++qp) {
    int qt[3];
    local_tuple(d, qp, 3, qt);
    double xq[3] = {0, 0, 0}, W = 1.0;
    for (int a = 0; a < d; ++a) {
      xq[a] = lo[a] + h[a] * kGaussX[qt[a]];
      W *= kGaussW[qt[a]] * h[a];
    }
    const double eta = viscosity(O.P, xq);
    double fq[3];
    forcing(O.P, fkind, xq, fq);
    double phi[8], grad[8][3];
    for (int A = 0; A < E.nl; ++A) {
      int at[3];
      local_tuple(d, A, 2, at);
      double p = 1.0;
      for (int a = 0; a < d; ++a) p *= q1(at[a], kGaussX[qt[a]]);
      phi[A] = p;
      for (int k = 0; k < d; ++k) {
        double gk = (at[k] == 0 ? -1.0 : 1.0) / h[k];
        for (int m = 0; m < d; ++m)
          if (m != k) gk *= q1(at[m], kGaussX[qt[m]]);
        grad[A][k] = gk;
      }
    }
    for (int A = 0; A < E.nl; ++A) {
      for (int A2 = 0; A2 < E.nl; ++A2) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += grad[A][k] * grad[A2][k];
        E.K[A][A2] += W * eta * s;
        E.C[A][A2] += -O.P.beta * diam2 * W * s;
      }
      for (int cc = 0; cc < d; ++cc) {
        for (int b = 0; b < E.nv; ++b) E.B[cc][A][b] += -W * phi[b] * grad[A][cc];
        E.F[A][cc] += W * fq[cc] * phi[A];
      }
    }
  }
}

// Position of column j in CSR row i (binary search); -1 if absent.
int64_t find_col(const Level& L, int64_t i, int64_t j) {
  auto b = L.ci.begin() + L.rp[i], e = L.ci.begin() + L.rp[i + 1];
  auto it = std::lower_bound(b, e, j);
  if (it == e || *it != j) return -1;
  return it - L.ci.begin();
}

// ---------------------------------------------------------------------------
// Numbering (all DoFs, Dirichlet included, live in x):
//   Q2 node I = (I_0, I_1[, I_2]) in [0,2N]^d, id = I_0 + (2N+1)(I_1 + (2N+1) I_2)
//   velocity DoF = d*id + c ; pressure vertex v, id_v = v_0 + (N+1)(v_1 + ...),
//   pressure DoF = n_u + id_v.
void init_level(const Oracle& O, Level& L) {
  const int d = L.dim;
  L.M = L.q * L.N + 1;
  L.nnode = 1;
  int64_t nvert = 1;
  for (int a = 0; a < d; ++a) { L.nnode *= L.M; nvert *= (L.N + 1); }
  L.n_u = d * L.nnode;
  L.n_p = nvert;
  L.n = L.n_u + L.n_p;
  L.dir.assign(L.n, 0);
  L.g.assign(L.n, 0.0);
  for (int64_t id = 0; id < L.nnode; ++id) {
    int64_t I[3];
    node_of(L, id, I);
    if (!node_on_boundary(L, I)) continue;
    double x[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) x[a] = node_coord(L, a, I[a]);
    const bool top = I[d - 1] == L.q * L.N;
    for (int c = 0; c < d; ++c) {
      L.dir[d * id + c] = 1;
      L.g[d * id + c] = boundary_value(O.P, x, top, c);
    }
  }
}

// Structural sparsity: a velocity row (I,c) couples to (J,c) for every node J
// and to p_v for every vertex v of a cell containing I; a pressure row v couples
// to (J,c') for every node J of a cell containing v; a Dirichlet row is the
// identity row.
void build_pattern(Level& L) {
  const int d = L.dim;
  L.rp.assign(L.n + 1, 0);
  std::vector<std::vector<int64_t>> rows(L.n);
  for (int64_t i = 0; i < L.n; ++i) {
    std::vector<int64_t>& cols = rows[i];
    if (i < L.n_u) {
      if (L.dir[i]) { cols.push_back(i); continue; }
      const int64_t id = i / d, comp = i % d;
      int64_t I[3];
      node_of(L, id, I);
      int64_t cl[3][2];
      int cnt[3] = {1, 1, 1};
      for (int a = 0; a < d; ++a) cnt[a] = cells_of_node(I[a], L.N, cl[a]);
      tensor_loop(d, cnt, [&](const int* k) {
        int64_t c[3];
        for (int a = 0; a < d; ++a) c[a] = cl[a][k[a]];
        int c3[3] = {3, 3, 3}, c2[3] = {2, 2, 2};
        tensor_loop(d, c3, [&](const int* t) {
          int64_t J[3];
          for (int a = 0; a < d; ++a) J[a] = 2 * c[a] + t[a];
          cols.push_back(d * node_id(L, J) + comp);
        });
        tensor_loop(d, c2, [&](const int* t) {
          int64_t v[3];
          for (int a = 0; a < d; ++a) v[a] = c[a] + t[a];
          cols.push_back(L.n_u + vert_id(L, v));
        });
      });
    } else {
      int64_t v[3];
      vert_of(L, i - L.n_u, v);
      int64_t cl[3][2];
      int cnt[3] = {1, 1, 1};
      for (int a = 0; a < d; ++a) cnt[a] = cells_of_vertex(v[a], L.N, cl[a]);
      tensor_loop(d, cnt, [&](const int* k) {
        int64_t c[3];
        for (int a = 0; a < d; ++a) c[a] = cl[a][k[a]];
        int c3[3] = {3, 3, 3};
        tensor_loop(d, c3, [&](const int* t) {
          int64_t J[3];
          for (int a = 0; a < d; ++a) J[a] = 2 * c[a] + t[a];
          for (int cc = 0; cc < d; ++cc) cols.push_back(d * node_id(L, J) + cc);
        });
      });
    }
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
  }
  for (int64_t i = 0; i < L.n; ++i) L.rp[i + 1] = L.rp[i] + (int64_t)rows[i].size();
  L.ci.resize(L.rp[L.n]);
  L.va.assign(L.rp[L.n], 0.0);
  for (int64_t i = 0; i < L.n; ++i) std::copy(rows[i].begin(), rows[i].end(), L.ci.begin() + L.rp[i]);
}

// Structural sparsity of the Q1-Q1 operator (velocity nodes are the vertices):
// a velocity row (v,c) couples to (w,c) and to p_w, and a pressure row v to
// (w,c') for every c' and to p_w, for every vertex w of a cell containing v
// (the p_w of a pressure row carry the stabilisation C); Dirichlet rows are
// identity rows.
void build_pattern_q1(Level& L) {
  const int d = L.dim;
  L.rp.assign(L.n + 1, 0);
  std::vector<std::vector<int64_t>> rows(L.n);
  for (int64_t i = 0; i < L.n; ++i) {
    std::vector<int64_t>& cols = rows[i];
    if (i < L.n_u && L.dir[i]) { cols.push_back(i); continue; }
    const bool vel = i < L.n_u;
    int64_t v[3];
    vert_of(L, vel ? i / d : i - L.n_u, v);
    int64_t cl[3][2];
    int cnt[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) cnt[a] = cells_of_vertex(v[a], L.N, cl[a]);
    tensor_loop(d, cnt, [&](const int* k) {
      int c2[3] = {2, 2, 2};
      tensor_loop(d, c2, [&](const int* t) {
        int64_t w[3];
        for (int a = 0; a < d; ++a) w[a] = cl[a][k[a]] + t[a];
        const int64_t id = vert_id(L, w);
        if (vel) {
          cols.push_back(d * id + i % d);
        } else {
          for (int cc = 0; cc < d; ++cc) cols.push_back(d * id + cc);
        }
        cols.push_back(L.n_u + id);
      });
    });
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
  }
  for (int64_t i = 0; i < L.n; ++i) L.rp[i + 1] = L.rp[i] + (int64_t)rows[i].size();
  L.ci.resize(L.rp[L.n]);
  L.va.assign(L.rp[L.n], 0.0);
  for (int64_t i = 0; i < L.n; ++i) std::copy(rows[i].begin(), rows[i].end(), L.ci.begin() + L.rp[i]);
}

// Element-by-element assembly of the stabilised Q1-Q1 operator (Eqs. 7-8).
void assemble_q1(const Oracle& O, Level& L) {
  const int d = L.dim;
  int cnt[3] = {L.N, L.N, L.N};
  Elem E;
  tensor_loop(d, cnt, [&](const int* ci) {
    int64_t c[3] = {ci[0], ci[1], ci[2]};
    element_q1(O, L, c, 0, E);
    int64_t gn[8];
    for (int A = 0; A < E.nl; ++A) {
      int at[3];
      local_tuple(d, A, 2, at);
      int64_t w[3];
      for (int a = 0; a < d; ++a) w[a] = c[a] + at[a];
      gn[A] = vert_id(L, w);
    }
    for (int A = 0; A < E.nl; ++A) {
      for (int cc = 0; cc < d; ++cc) {
        const int64_t row = d * gn[A] + cc;
        if (!L.dir[row]) {
          for (int A2 = 0; A2 < E.nl; ++A2) L.va[find_col(L, row, d * gn[A2] + cc)] += E.K[A][A2];
          for (int b = 0; b < E.nv; ++b) L.va[find_col(L, row, L.n_u + gn[b])] += E.B[cc][A][b];
        }
        for (int b = 0; b < E.nv; ++b) L.va[find_col(L, L.n_u + gn[b], row)] += E.B[cc][A][b];
      }
    }
    for (int a = 0; a < E.nv; ++a)
      for (int b = 0; b < E.nv; ++b) L.va[find_col(L, L.n_u + gn[a], L.n_u + gn[b])] += E.C[a][b];
  });
  for (int64_t i = 0; i < L.n_u; ++i)
    if (L.dir[i]) L.va[find_col(L, i, i)] = 1.0;
}

// Standard element-by-element assembly of L (Eq. 7 on Q2-Q1, C = 0).
void assemble(const Oracle& O, Level& L) {
  const int d = L.dim;
  int cnt[3] = {L.N, L.N, L.N};
  Elem E;
  tensor_loop(d, cnt, [&](const int* ci) {
    int64_t c[3] = {ci[0], ci[1], ci[2]};
    element(O, L, c, 0, E);
    int64_t gn[27], gv[8];
    for (int A = 0; A < E.nl; ++A) {
      int at[3];
      local_tuple(d, A, 3, at);
      int64_t J[3];
      for (int a = 0; a < d; ++a) J[a] = 2 * c[a] + at[a];
      gn[A] = node_id(L, J);
    }
    for (int b = 0; b < E.nv; ++b) {
      int bt[3];
      local_tuple(d, b, 2, bt);
      int64_t v[3];
      for (int a = 0; a < d; ++a) v[a] = c[a] + bt[a];
      gv[b] = L.n_u + vert_id(L, v);
    }
    for (int A = 0; A < E.nl; ++A) {
      for (int cc = 0; cc < d; ++cc) {
        const int64_t row = d * gn[A] + cc;
        if (!L.dir[row]) {
          for (int A2 = 0; A2 < E.nl; ++A2) L.va[find_col(L, row, d * gn[A2] + cc)] += E.K[A][A2];
          for (int b = 0; b < E.nv; ++b) L.va[find_col(L, row, gv[b])] += E.B[cc][A][b];
        }
        for (int b = 0; b < E.nv; ++b) L.va[find_col(L, gv[b], row)] += E.B[cc][A][b];
      }
    }
  });
  for (int64_t i = 0; i < L.n_u; ++i)
    if (L.dir[i]) L.va[find_col(L, i, i)] = 1.0;
}

// Canonical nested interpolation from coarse level C into fine level F:
// a fine Q2 node takes the value of the coarse piecewise-quadratic function at
// its position (1-D Lagrange weights of the coarse cell that contains it,
// tensorised); a fine pressure vertex takes the coarse piecewise-bilinear
// (trilinear) value, and so does a fine Q1 velocity node.  Rows of fine
// Dirichlet DoFs are empty.
void build_prolongation(const Level& C, Level& F) {
  const int d = F.dim;
  F.Prp.assign(F.n + 1, 0);
  std::vector<std::vector<std::pair<int64_t, double>>> rows(F.n);
  // per-axis weights for a fine Q2 node index I: coarse nodes and weights
  auto q2w = [&](int a, int64_t I, int64_t* K, double* w) {
    const double x = node_coord(F, a, I);
    int64_t k = I / 4;
    if (k > C.N - 1) k = C.N - 1;
    const double t = (x - C.xv[a][k]) / (C.xv[a][k + 1] - C.xv[a][k]);
    for (int j = 0; j < 3; ++j) { K[j] = 2 * k + j; w[j] = q2(j, t); }
  };
  auto q1w = [&](int a, int64_t v, int64_t* K, double* w) {
    const double x = F.xv[a][v];
    int64_t k = v / 2;
    if (k > C.N - 1) k = C.N - 1;
    const double t = (x - C.xv[a][k]) / (C.xv[a][k + 1] - C.xv[a][k]);
    for (int j = 0; j < 2; ++j) { K[j] = k + j; w[j] = q1(j, t); }
  };
  for (int64_t id = 0; id < F.nnode; ++id) {
    int64_t I[3];
    node_of(F, id, I);
    int64_t K[3][3];
    double w[3][3];
    for (int a = 0; a < d; ++a) {
      if (F.q == 2) q2w(a, I[a], K[a], w[a]);
      else q1w(a, I[a], K[a], w[a]);
    }
    for (int cc = 0; cc < d; ++cc) {
      const int64_t row = d * id + cc;
      if (F.dir[row]) continue;
      int c3[3] = {F.q + 1, F.q + 1, F.q + 1};
      tensor_loop(d, c3, [&](const int* t) {
        int64_t J[3];
        double ww = 1.0;
        for (int a = 0; a < d; ++a) { J[a] = K[a][t[a]]; ww *= w[a][t[a]]; }
        if (ww != 0.0) rows[row].push_back({d * node_id(C, J) + cc, ww});
      });
    }
  }
  for (int64_t vid = 0; vid < F.n_p; ++vid) {
    int64_t v[3];
    vert_of(F, vid, v);
    int64_t K[3][2];
    double w[3][2];
    for (int a = 0; a < d; ++a) q1w(a, v[a], K[a], w[a]);
    int c2[3] = {2, 2, 2};
    tensor_loop(d, c2, [&](const int* t) {
      int64_t J[3];
      double ww = 1.0;
      for (int a = 0; a < d; ++a) { J[a] = K[a][t[a]]; ww *= w[a][t[a]]; }
      if (ww != 0.0) rows[F.n_u + vid].push_back({C.n_u + vert_id(C, J), ww});
    });
  }
  for (int64_t i = 0; i < F.n; ++i) {
    std::sort(rows[i].begin(), rows[i].end());
    F.Prp[i + 1] = F.Prp[i] + (int64_t)rows[i].size();
  }
  F.Pci.resize(F.Prp[F.n]);
  F.Pva.resize(F.Prp[F.n]);
  for (int64_t i = 0; i < F.n; ++i)
    for (size_t k = 0; k < rows[i].size(); ++k) {
      F.Pci[F.Prp[i] + k] = rows[i][k].first;
      F.Pva[F.Prp[i] + k] = rows[i][k].second;
    }
}

// ---------------------------------------------------------------------------
// Dense LU with partial pivoting (row swap to the largest |pivot|, the lowest
// row index wins ties).  a is n x n row-major, overwritten by L\U; returns
// false when a pivot is below 1e-14 * max|a|.
bool lu_factor(std::vector<double>& a, int64_t n, std::vector<int64_t>& piv) {
  piv.resize(n);
  double amax = 0.0;
  for (double v : a) amax = std::max(amax, std::fabs(v));
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = k;
    double best = std::fabs(a[k * n + k]);
    for (int64_t i = k + 1; i < n; ++i)
      if (std::fabs(a[i * n + k]) > best) { best = std::fabs(a[i * n + k]); p = i; }
    piv[k] = p;
    if (best <= 1e-14 * amax) return false;
    if (p != k)
      for (int64_t j = 0; j < n; ++j) std::swap(a[k * n + j], a[p * n + j]);
    for (int64_t i = k + 1; i < n; ++i) {
      const double l = a[i * n + k] / a[k * n + k];
      a[i * n + k] = l;
      for (int64_t j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return true;
}
// Solve (LU) z = rhs in place.
void lu_solve(const std::vector<double>& a, int64_t n, const std::vector<int64_t>& piv, double* z) {
  for (int64_t k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(z[k], z[piv[k]]);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < i; ++j) z[i] -= a[i * n + j] * z[j];
  for (int64_t i = n - 1; i >= 0; --i) {
    for (int64_t j = i + 1; j < n; ++j) z[i] -= a[i * n + j] * z[j];
    z[i] /= a[i * n + i];
  }
}

// ---------------------------------------------------------------------------
// Subdomains (Sec. 3): S_i = {p_i} u {velocity DoFs of every velocity node of
// every cell containing vertex i} minus Dirichlet DoFs, sorted ascending.
// Ownership (the restricted set of Eq. 13): on Q1-Q1 the velocity DoFs of
// vertex i itself (the paper's rule); extended to Q2, a velocity DoF at node I
// is owned by vertex floor(I/2) (componentwise), i.e. a vertex node by its own
// vertex and an edge/face/cell node by the lowest vertex of its entity; p_i is
// owned by i; Dirichlet DoFs have no owner.
void build_patches(Level& L) {
  const int d = L.dim;
  L.poff.assign(L.n_p + 1, 0);
  L.pdof.clear();
  L.owner.assign(L.n, -1);
  for (int64_t id = 0; id < L.nnode; ++id) {
    int64_t I[3], v[3];
    node_of(L, id, I);
    for (int a = 0; a < d; ++a) v[a] = I[a] / L.q;
    for (int c = 0; c < d; ++c)
      if (!L.dir[d * id + c]) L.owner[d * id + c] = vert_id(L, v);
  }
  for (int64_t p = 0; p < L.n_p; ++p) L.owner[L.n_u + p] = p;
  for (int64_t p = 0; p < L.n_p; ++p) {
    int64_t v[3];
    vert_of(L, p, v);
    std::vector<int64_t> s;
    int64_t cl[3][2];
    int cnt[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) cnt[a] = cells_of_vertex(v[a], L.N, cl[a]);
    tensor_loop(d, cnt, [&](const int* k) {
      int c3[3] = {L.q + 1, L.q + 1, L.q + 1};
      tensor_loop(d, c3, [&](const int* t) {
        int64_t J[3];
        for (int a = 0; a < d; ++a) J[a] = L.q * cl[a][k[a]] + t[a];
        for (int c = 0; c < d; ++c) {
          int64_t dof = d * node_id(L, J) + c;
          if (!L.dir[dof]) s.push_back(dof);
        }
      });
    });
    s.push_back(L.n_u + p);
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
    L.pdof.insert(L.pdof.end(), s.begin(), s.end());
    L.poff[p + 1] = (int64_t)L.pdof.size();
  }
}

void fill_owned(Level& L) {
  const int64_t np = (int64_t)L.poff.size() - 1;
  L.owned.assign(np, {});
  for (int64_t p = 0; p < np; ++p)
    for (int64_t k = L.poff[p]; k < L.poff[p + 1]; ++k)
      if (L.owner[L.pdof[k]] == p) L.owned[p].push_back((int)(k - L.poff[p]));
}

// L_i = R_i L R_i^T as a dense row-major matrix.
void local_matrix(const Level& L, int64_t p, std::vector<double>& Li) {
  const int64_t b = L.poff[p], ni = L.poff[p + 1] - b;
  Li.assign(ni * ni, 0.0);
  for (int64_t r = 0; r < ni; ++r) {
    const int64_t row = L.pdof[b + r];
    for (int64_t c = 0; c < ni; ++c) {
      int64_t k = find_col(L, row, L.pdof[b + c]);
      if (k >= 0) Li[r * ni + c] = L.va[k];
    }
  }
}

// Rows of L_i^{-1}.  Row j of L_i^{-1} solves L_i^T y = e_j, so the transpose
// is factorised and solved for the wanted unit vectors.  all_rows selects the
// full inverse (AV, MV) instead of the owned rows (RAV).
bool inverse_rows(const Level& L, int64_t p, bool all_rows, std::vector<double>& out) {
  std::vector<double> Li, T;
  local_matrix(L, p, Li);
  const int64_t ni = L.poff[p + 1] - L.poff[p];
  T.resize(ni * ni);
  for (int64_t r = 0; r < ni; ++r)
    for (int64_t c = 0; c < ni; ++c) T[c * ni + r] = Li[r * ni + c];
  std::vector<int64_t> piv;
  if (!lu_factor(T, ni, piv)) return false;
  std::vector<int> rows;
  if (all_rows)
    for (int r = 0; r < ni; ++r) rows.push_back(r);
  else
    rows = L.owned[p];
  out.assign(rows.size() * ni, 0.0);
  std::vector<double> z(ni);
  for (size_t k = 0; k < rows.size(); ++k) {
    std::fill(z.begin(), z.end(), 0.0);
    z[rows[k]] = 1.0;
    lu_solve(T, ni, piv, z.data());
    std::copy(z.begin(), z.end(), out.begin() + k * ni);
  }
  return true;
}

// ---------------------------------------------------------------------------
// Reduced-precision emulation: round-to-nearest-even of a double to a binary
// format with p significand bits, minimum normal exponent emin, largest finite
// value vmax (saturating).
double round_format(double v, int p, int emin, double vmax) {
  if (v == 0.0 || !std::isfinite(v)) return v;
  int E;
  std::frexp(v, &E);  // |v| = m 2^E, m in [0.5,1): leading bit has exponent E-1
  int e = E - 1;
  if (e < emin) e = emin;
  const double quantum = std::ldexp(1.0, e - (p - 1));
  double q = std::nearbyint(v / quantum) * quantum;
  if (q > vmax) q = vmax;
  if (q < -vmax) q = -vmax;
  return q;
}
double fmt_round(int prec, double v) {
  if (prec == 1) return round_format(v, 24, -126, 3.4028234663852886e38);
  if (prec == 2) return round_format(v, 8, -126, 3.3895313892515355e38);
  if (prec == 3) return round_format(v, 4, -6, 448.0);
  return v;
}
// Per-row scale: 1 for fp32/bf16; max|row|/448 rounded to fp32 for fp8 e4m3.
double fmt_scale(int prec, const double* row, int64_t n) {
  if (prec != 3) return 1.0;
  double m = 0.0;
  for (int64_t k = 0; k < n; ++k) m = std::max(m, std::fabs(row[k]));
  if (m == 0.0) return 1.0;
  return (double)(float)(m / 448.0);
}

// Factored storage of the owned rows (prec 5: fp32, 6: bf16).  The local
// system of Eq. 11 has the saddle-point form L_i = [A b; b^T c] (one pressure
// DoF, the last in sorted order; c = 0 on Q2-Q1, the diagonal entry of the
// stabilisation of Eq. 8 on Q1-Q1), so with w = A^{-1} b and s = c - b^T w
//   L_i^{-1} = [A^{-1} + w w^T / s,  -w / s;  -w^T / s,  1 / s].
// The owned rows of A^{-1}, w and 1/s are rounded to the format, then the owned
// rows of L_i^{-1} are rebuilt from the rounded values by that formula in fp64.
bool factored_rows(const Level& L, int64_t p, int fmt, std::vector<double>& out) {
  std::vector<double> Li;
  local_matrix(L, p, Li);
  const int64_t ni = L.poff[p + 1] - L.poff[p], nv = ni - 1;
  std::vector<double> T(nv * nv), w(nv);
  for (int64_t r = 0; r < nv; ++r) {
    w[r] = Li[r * ni + nv];
    for (int64_t c = 0; c < nv; ++c) T[c * nv + r] = Li[r * ni + c];  // A^T
  }
  std::vector<int64_t> piv;
  if (!lu_factor(T, nv, piv)) return false;
  std::vector<double> Tt(nv * nv);  // A itself, for w = A^{-1} b
  for (int64_t r = 0; r < nv; ++r)
    for (int64_t c = 0; c < nv; ++c) Tt[r * nv + c] = Li[r * ni + c];
  std::vector<int64_t> piv2;
  if (!lu_factor(Tt, nv, piv2)) return false;
  lu_solve(Tt, nv, piv2, w.data());
  double s = Li[nv * ni + nv];
  for (int64_t r = 0; r < nv; ++r) s -= Li[nv * ni + r] * w[r];
  if (s == 0.0) return false;
  const double sig = fmt_round(fmt, 1.0 / s);
  std::vector<double> rw(nv);
  for (int64_t r = 0; r < nv; ++r) rw[r] = fmt_round(fmt, w[r]);
  const std::vector<int>& rows = L.owned[p];
  out.assign(rows.size() * ni, 0.0);
  std::vector<double> z(nv);
  for (size_t k = 0; k < rows.size(); ++k) {
    double* o = &out[k * ni];
    const int j = rows[k];
    if (j == nv) {  // pressure row
      for (int64_t c = 0; c < nv; ++c) o[c] = -rw[c] * sig;
      o[nv] = sig;
      continue;
    }
    std::fill(z.begin(), z.end(), 0.0);
    z[j] = 1.0;
    lu_solve(T, nv, piv, z.data());  // row j of A^{-1}
    for (int64_t c = 0; c < nv; ++c) o[c] = fmt_round(fmt, z[c]) + rw[j] * rw[c] * sig;
    o[nv] = -rw[j] * sig;
  }
  return true;
}

void quantise(Oracle& O, Level& L) {
  const int64_t np = (int64_t)L.poff.size() - 1;
  L.qinv.assign(np, {});
  L.qscale.assign(np, {});
  if (O.prec == 0) return;
  if (O.prec >= 5) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int64_t p = 0; p < np; ++p) {
      factored_rows(L, p, O.prec - 4, L.qinv[p]);
      L.qscale[p].assign(L.owned[p].size(), 1.0);
    }
    return;
  }
  for (int64_t p = 0; p < np; ++p) {
    const int64_t ni = L.poff[p + 1] - L.poff[p];
    const int64_t nr = (int64_t)L.inv[p].size() / std::max<int64_t>(ni, 1);
    L.qinv[p].resize(L.inv[p].size());
    L.qscale[p].resize(nr);
    for (int64_t r = 0; r < nr; ++r) {
      const double* row = &L.inv[p][r * ni];
      const double s = fmt_scale(O.prec, row, ni);
      L.qscale[p][r] = s;
      for (int64_t k = 0; k < ni; ++k) L.qinv[p][r * ni + k] = fmt_round(O.prec, row[k] / s);
    }
  }
}

// ---------------------------------------------------------------------------
// r = b - L x on free rows, 0 on Dirichlet rows (Eq. 10).
void residual(const Level& L, const double* x, const double* b, double* r) {
  for (int64_t i = 0; i < L.n; ++i) {
    if (L.dir[i]) { r[i] = 0.0; continue; }
    double s = b[i];
    for (int64_t k = L.rp[i]; k < L.rp[i + 1]; ++k) s -= L.va[k] * x[L.ci[k]];
    r[i] = s;
  }
}

// y = row block (nr x ni) times rloc, in fp64, or emulating the reduced-precision
// apply: fp32 products of the quantised entry and the fp32-rounded residual,
// accumulated in fp32 in ascending column order, then scaled by the fp32 row scale.
void apply_rows(const Oracle& O, const Level& L, int64_t p, const double* rloc, int64_t ni, double* y) {
  const std::vector<double>& R = L.inv[p];
  const int64_t nr = (int64_t)R.size() / std::max<int64_t>(ni, 1);
  for (int64_t j = 0; j < nr; ++j) {
    if (O.prec == 0 || O.prec >= 5) {
      const std::vector<double>& M = O.prec == 0 ? R : L.qinv[p];
      double s = 0.0;
      for (int64_t k = 0; k < ni; ++k) s += M[j * ni + k] * rloc[k];
      y[j] = s;
    } else {
      float s = 0.0f;
      for (int64_t k = 0; k < ni; ++k) s += (float)L.qinv[p][j * ni + k] * (float)rloc[k];
      y[j] = (double)(s * (float)L.qscale[p][j]);
    }
  }
}

// One smoothing step x <- x + S (b - L x) for the chosen Vanka variant.
void smooth(Oracle& O, Level& L, double* x, const double* b) {
  const int64_t np = (int64_t)L.poff.size() - 1;
  std::vector<double> r(L.n), rloc, y;
  if (O.kind == 0 || O.kind == 1) {
    residual(L, x, b, r.data());
    std::vector<double> xn(x, x + L.n);
    // The subdomain corrections all use the same residual r.  RAV (Eq. 13)
    // writes only owned DoFs, which belong to one subdomain each, so its
    // subdomains are independent; AV (Eq. 12) adds overlapping corrections to
    // shared DoFs and stays in ascending subdomain order.
#pragma omp parallel for schedule(dynamic, 64) num_threads(O.kind == 0 ? g_threads : 1) private(rloc, y)
    for (int64_t p = 0; p < np; ++p) {
      const int64_t b0 = L.poff[p], ni = L.poff[p + 1] - b0;
      rloc.resize(ni);
      for (int64_t k = 0; k < ni; ++k) rloc[k] = r[L.pdof[b0 + k]];
      y.assign(O.kind == 0 ? L.owned[p].size() : ni, 0.0);
      apply_rows(O, L, p, rloc.data(), ni, y.data());
      if (O.kind == 0) {  // Eq. 13: only the owned DoFs take the correction
        for (size_t j = 0; j < L.owned[p].size(); ++j) xn[L.pdof[b0 + L.owned[p][j]]] += L.omega[p] * y[j];
      } else {            // Eq. 12: every DoF of the subdomain takes it
        for (int64_t k = 0; k < ni; ++k) xn[L.pdof[b0 + k]] += L.omega[p] * y[k];
      }
    }
    std::copy(xn.begin(), xn.end(), x);
    return;
  }
  // Multiplicative (Eq. 11 as a sequential sweep, residual refreshed per
  // subdomain as in Eq. 15, read as r_m = b_m - sum_k L_mk x_k).
  std::vector<int64_t> order(np);
  for (int64_t p = 0; p < np; ++p) order[p] = p;
  if (O.kind == 3) {  // coloured order: colour = sum_a (v_a mod 4) 4^a, ascending
    auto colour = [&](int64_t p) {
      int64_t v[3];
      vert_of(L, p, v);
      int64_t c = 0, m = 1;
      for (int a = 0; a < L.dim; ++a) { c += (v[a] % 4) * m; m *= 4; }
      return c;
    };
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b2) { return colour(a) < colour(b2); });
  }
  for (int64_t oi = 0; oi < np; ++oi) {
    const int64_t p = order[oi];
    const int64_t b0 = L.poff[p], ni = L.poff[p + 1] - b0;
    rloc.resize(ni);
    for (int64_t k = 0; k < ni; ++k) {
      const int64_t m = L.pdof[b0 + k];
      double s = b[m];
      for (int64_t q = L.rp[m]; q < L.rp[m + 1]; ++q) s -= L.va[q] * x[L.ci[q]];
      rloc[k] = s;
    }
    y.assign(ni, 0.0);
    apply_rows(O, L, p, rloc.data(), ni, y.data());
    for (int64_t k = 0; k < ni; ++k) x[L.pdof[b0 + k]] += L.omega[p] * y[k];
  }
}

// Coarse solve: LU of the bordered system [L e_p; e_p^T 0], e_p = 1 on the
// pressure DoFs, which is non-singular although L has the constant pressure in
// its kernel; the solution has zero pressure sum.
bool coarse_factor(Level& L) {
  const int64_t m = L.n + 1;
  L.clu.assign(m * m, 0.0);
  for (int64_t i = 0; i < L.n; ++i)
    for (int64_t k = L.rp[i]; k < L.rp[i + 1]; ++k) L.clu[i * m + L.ci[k]] = L.va[k];
  for (int64_t i = L.n_u; i < L.n; ++i) {
    L.clu[i * m + L.n] = 1.0;
    L.clu[L.n * m + i] = 1.0;
  }
  return lu_factor(L.clu, m, L.cpiv);
}
void coarse_solve(Level& L, const double* b, double* x) {
  const int64_t m = L.n + 1;
  if (L.clu.empty() && !coarse_factor(L)) {  // factorised on first use
    std::fill(x, x + L.n, std::nan(""));
    return;
  }
  std::vector<double> z(m, 0.0);
  for (int64_t i = 0; i < L.n; ++i) z[i] = L.dir[i] ? 0.0 : b[i];
  lu_solve(L.clu, m, L.cpiv, z.data());
  for (int64_t i = 0; i < L.n; ++i) x[i] = z[i];
}

// x_f += P x_c (fine Dirichlet rows of P are empty).
void prolong_add(const Level& F, const double* xc, double* xf) {
  for (int64_t i = 0; i < F.n; ++i)
    for (int64_t k = F.Prp[i]; k < F.Prp[i + 1]; ++k) xf[i] += F.Pva[k] * xc[F.Pci[k]];
}
// b_c = P^T r_f, then 0 on coarse Dirichlet rows.
void restrict_(const Level& F, const Level& C, const double* rf, double* bc) {
  std::fill(bc, bc + C.n, 0.0);
  for (int64_t i = 0; i < F.n; ++i)
    for (int64_t k = F.Prp[i]; k < F.Prp[i + 1]; ++k) bc[F.Pci[k]] += F.Pva[k] * rf[i];
  for (int64_t i = 0; i < C.n; ++i)
    if (C.dir[i]) bc[i] = 0.0;
}

// V(nu1, nu2) cycle on level l (Sec. 2, Fig. 1).
void vcycle(Oracle& O, int l, double* x, const double* b, int nu1, int nu2) {
  Level& L = O.lev[l];
  if (l == 0) {
    std::vector<double> r(L.n), e(L.n);
    residual(L, x, b, r.data());
    coarse_solve(L, r.data(), e.data());
    for (int64_t i = 0; i < L.n; ++i) x[i] += e[i];
    return;
  }
  for (int s = 0; s < nu1; ++s) smooth(O, L, x, b);
  Level& C = O.lev[l - 1];
  std::vector<double> r(L.n), bc(C.n), xc(C.n, 0.0);
  residual(L, x, b, r.data());
  restrict_(L, C, r.data(), bc.data());
  vcycle(O, l - 1, xc.data(), bc.data(), nu1, nu2);
  prolong_add(L, xc.data(), x);
  for (int s = 0; s < nu2; ++s) smooth(O, L, x, b);
}

double norm2(const std::vector<double>& v) {
  double s = 0.0;
  for (double a : v) s += a * a;
  return std::sqrt(s);
}

}  // namespace

// =============================================================================
// C interface (ctypes).  Level index 0 is the coarsest.
extern "C" {

// coords: dim*(N+1) vertex coordinates of the finest level, axis-major; NULL = uniform on [0,1].
// blobs: nblobs*5 (cx, cy, cz, rho, s).  elem: 0 Q2-Q1, 1 stabilised Q1-Q1 with
// constant beta (Eq. 8).
void* orc_create_elem(int dim, int N, int nlev, const double* coords, double eta0, int nblobs,
                      const double* blobs, int bc, int elem, double beta) {
  Oracle* O = new Oracle();
  O->P.dim = dim;
  O->P.eta0 = eta0;
  O->P.bc = bc;
  O->P.elem = elem;
  O->P.beta = elem == 1 ? beta : 0.0;
  O->P.blobs.assign(blobs, blobs + 5 * nblobs);
  O->lev.resize(nlev);
  for (int l = nlev - 1; l >= 0; --l) {
    Level& L = O->lev[l];
    L.dim = dim;
    L.q = elem == 1 ? 1 : 2;
    const int stride = 1 << (nlev - 1 - l);
    L.N = N / stride;
    for (int a = 0; a < dim; ++a) {
      L.xv[a].resize(L.N + 1);
      for (int k = 0; k <= L.N; ++k)
        L.xv[a][k] = coords ? coords[a * (N + 1) + k * stride] : (double)(k * stride) / N;
    }
    init_level(*O, L);
    if (l != nlev - 1) std::fill(L.g.begin(), L.g.end(), 0.0);
    if (L.q == 1) {
      build_pattern_q1(L);
      assemble_q1(*O, L);
    } else {
      build_pattern(L);
      assemble(*O, L);
    }
  }
  for (int l = 1; l < nlev; ++l) build_prolongation(O->lev[l - 1], O->lev[l]);
  return O;
}
void* orc_create(int dim, int N, int nlev, const double* coords, double eta0, int nblobs,
                 const double* blobs, int bc) {
  return orc_create_elem(dim, N, nlev, coords, eta0, nblobs, blobs, bc, 0, 0.0);
}

void orc_destroy(void* h) { delete (Oracle*)h; }
// 0, or -3 when the bordered coarse system is singular (checked by factorising it).
int orc_error(void* h) {
  Level& C = ((Oracle*)h)->lev[0];
  if (C.clu.empty() && !coarse_factor(C)) return -3;
  return ((Oracle*)h)->err;
}

// what: 0 n_u, 1 n_p, 2 n, 3 nnz, 4 N, 5 number of subdomains, 6 total subdomain DoFs,
//       7 prolongation nnz
long long orc_count(void* h, int l, int what) {
  const Level& L = ((Oracle*)h)->lev[l];
  switch (what) {
    case 0: return L.n_u;
    case 1: return L.n_p;
    case 2: return L.n;
    case 3: return (long long)L.ci.size();
    case 4: return L.N;
    case 5: return L.poff.empty() ? 0 : (long long)L.poff.size() - 1;
    case 6: return (long long)L.pdof.size();
    case 7: return (long long)L.Pci.size();
  }
  return -1;
}

void orc_get_csr(void* h, int l, int64_t* rp, int64_t* ci, double* va) {
  const Level& L = ((Oracle*)h)->lev[l];
  std::copy(L.rp.begin(), L.rp.end(), rp);
  std::copy(L.ci.begin(), L.ci.end(), ci);
  std::copy(L.va.begin(), L.va.end(), va);
}
void orc_get_prolongation(void* h, int l, int64_t* rp, int64_t* ci, double* va) {
  const Level& L = ((Oracle*)h)->lev[l];
  std::copy(L.Prp.begin(), L.Prp.end(), rp);
  std::copy(L.Pci.begin(), L.Pci.end(), ci);
  std::copy(L.Pva.begin(), L.Pva.end(), va);
}
void orc_get_dirichlet(void* h, int l, uint8_t* mask, double* g) {
  const Level& L = ((Oracle*)h)->lev[l];
  if (mask) std::copy(L.dir.begin(), L.dir.end(), mask);
  if (g) std::copy(L.g.begin(), L.g.end(), g);
}

// Fine-level right-hand side: b_u = int v.f (3^d Gauss points), b_p = 0, b = g on Dirichlet rows.
void orc_rhs(void* h, int fkind, double* b) {
  Oracle& O = *(Oracle*)h;
  Level& L = O.lev.back();
  const int d = L.dim;
  std::fill(b, b + L.n, 0.0);
  int cnt[3] = {L.N, L.N, L.N};
  Elem E;
  tensor_loop(d, cnt, [&](const int* ci) {
    int64_t c[3] = {ci[0], ci[1], ci[2]};
    if (L.q == 1) element_q1(O, L, c, fkind, E);
    else element(O, L, c, fkind, E);
    for (int A = 0; A < E.nl; ++A) {
      int at[3];
      local_tuple(d, A, L.q + 1, at);
      int64_t J[3];
      for (int a = 0; a < d; ++a) J[a] = L.q * c[a] + at[a];
      const int64_t id = node_id(L, J);
      for (int cc = 0; cc < d; ++cc) b[d * id + cc] += E.F[A][cc];
    }
  });
  for (int64_t i = 0; i < L.n; ++i)
    if (L.dir[i]) b[i] = L.g[i];
}

// Threads of the subdomain loops (>= 1); returns the number in effect, which
// is 1 when the library was built without OpenMP.
int orc_set_threads(int n) {
#ifdef _OPENMP
  g_threads = n < 1 ? 1 : n;
#else
  (void)n;
  g_threads = 1;
#endif
  return g_threads;
}

// Viscosity at a point (so tests can check the coefficient field).
double orc_viscosity(void* h, const double* x) { return viscosity(((Oracle*)h)->P, x); }

// Builds subdomains, ownership and inverses on every level.
// kind: 0 RAV, 1 AV, 2 MV (lexicographic), 3 MV (4^d-coloured order).
// prec: 0 fp64, 1 fp32, 2 bf16, 3 fp8 e4m3 (stored inverse rows, fp32 accumulation);
// 5 fp32, 6 bf16 factored storage (rows rebuilt from rounded A^{-1}, w, 1/s; fp64 apply).
int orc_setup_smoother(void* h, int kind, double omega, int prec) {
  Oracle& O = *(Oracle*)h;
  O.kind = kind;
  O.prec = prec;
  for (size_t l = 1; l < O.lev.size(); ++l) {
    Level& L = O.lev[l];
    build_patches(L);
    fill_owned(L);
    const int64_t np = (int64_t)L.poff.size() - 1;
    L.inv.assign(np, {});
    L.omega.assign(np, omega);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads) reduction(|: bad)
    for (int64_t p = 0; p < np; ++p)
      if (!inverse_rows(L, p, kind != 0, L.inv[p])) bad = 1;
    if (bad) return -3;
    quantise(O, L);
  }
  return 0;
}

// Subdomain structure only (no inverses) on level l.
void orc_build_patches(void* h, int l) {
  Level& L = ((Oracle*)h)->lev[l];
  build_patches(L);
  fill_owned(L);
}

// Replaces the subdomains of level l (test use): npatch lists with offsets/dofs,
// owner per DoF (-1 = not owned).  Recomputes inverses for the current kind.
int orc_set_patches(void* h, int l, long long np, const int64_t* off, const int64_t* dofs, const int64_t* owner,
                    double omega) {
  Oracle& O = *(Oracle*)h;
  Level& L = O.lev[l];
  L.poff.assign(off, off + np + 1);
  L.pdof.assign(dofs, dofs + off[np]);
  L.owner.assign(owner, owner + L.n);
  fill_owned(L);
  L.inv.assign(np, {});
  L.omega.assign(np, omega);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads) reduction(|: bad)
  for (long long p = 0; p < np; ++p)
    if (!inverse_rows(L, p, O.kind != 0, L.inv[p])) bad = 1;
  if (bad) return -3;
  quantise(O, L);
  return 0;
}

void orc_set_omega(void* h, int l, const double* w) {
  Level& L = ((Oracle*)h)->lev[l];
  std::copy(w, w + L.omega.size(), L.omega.begin());
}

void orc_get_patches(void* h, int l, int64_t* off, int64_t* dofs, int64_t* owner) {
  const Level& L = ((Oracle*)h)->lev[l];
  std::copy(L.poff.begin(), L.poff.end(), off);
  std::copy(L.pdof.begin(), L.pdof.end(), dofs);
  std::copy(L.owner.begin(), L.owner.end(), owner);
}

// Owned-row block (RAV) or full inverse (AV/MV) of subdomain p, row-major over
// the sorted subdomain DoFs; the quantised values when prec != 0 and q != 0.
long long orc_get_inverse(void* h, int l, long long p, int q, double* out, double* scale) {
  const Level& L = ((Oracle*)h)->lev[l];
  const std::vector<double>& v = q ? L.qinv[p] : L.inv[p];
  if (out) std::copy(v.begin(), v.end(), out);
  if (scale && q) std::copy(L.qscale[p].begin(), L.qscale[p].end(), scale);
  return (long long)v.size();
}

// Owned rows of L_p^{-1} computed on demand (level l, subdomain p) without a full setup;
// needs orc_build_patches(l).  Returns the number of rows, or -3 for a singular L_p.
int orc_patch_rows(void* h, int l, long long p, double* out) {
  const Level& L = ((Oracle*)h)->lev[l];
  std::vector<double> rows;
  if (!inverse_rows(L, p, false, rows)) return -3;
  std::copy(rows.begin(), rows.end(), out);
  return (int)L.owned[p].size();
}

void orc_residual(void* h, int l, const double* x, const double* b, double* r) {
  residual(((Oracle*)h)->lev[l], x, b, r);
}
void orc_smooth(void* h, int l, double* x, const double* b, int steps) {
  Oracle& O = *(Oracle*)h;
  for (int s = 0; s < steps; ++s) smooth(O, O.lev[l], x, b);
}
void orc_restrict(void* h, int l, const double* rf, double* bc) {
  Oracle& O = *(Oracle*)h;
  restrict_(O.lev[l], O.lev[l - 1], rf, bc);
}
void orc_prolong_add(void* h, int l, const double* xc, double* xf) {
  prolong_add(((Oracle*)h)->lev[l], xc, xf);
}
void orc_coarse_solve(void* h, const double* b, double* x) { coarse_solve(((Oracle*)h)->lev[0], b, x); }
void orc_vcycle(void* h, double* x, const double* b, int nu1, int nu2) {
  Oracle& O = *(Oracle*)h;
  vcycle(O, (int)O.lev.size() - 1, x, b, nu1, nu2);
}

// Stationary multigrid: x <- V(nu1,nu2) until ||r||/||r0|| <= tol.
// hist[k] = ||r_k||/||r_0|| for k = 0..iters.  Returns iterations, or -5 if maxit reached.
int orc_solve(void* h, double* x, const double* b, double tol, int maxit, int nu1, int nu2, double* hist) {
  Oracle& O = *(Oracle*)h;
  Level& L = O.lev.back();
  std::vector<double> r(L.n);
  residual(L, x, b, r.data());
  const double r0 = norm2(r);
  hist[0] = 1.0;
  if (r0 == 0.0) return 0;
  for (int k = 1; k <= maxit; ++k) {
    vcycle(O, (int)O.lev.size() - 1, x, b, nu1, nu2);
    residual(L, x, b, r.data());
    hist[k] = norm2(r) / r0;
    if (!(hist[k] == hist[k])) return -7;
    if (hist[k] <= tol) return k;
  }
  return -5;
}

// FGMRES(m), right-preconditioned by one V-cycle from a zero guess, modified
// Gram-Schmidt, Givens rotations.  hist[k] = ||r_k||/||r_0|| after each inner
// iteration (true residual recomputed at restarts).  Returns total inner
// iterations, or -5 if maxit reached.
int orc_fgmres(void* h, double* x, const double* b, double tol, int maxit, int restart, int nu1, int nu2,
               double* hist) {
  Oracle& O = *(Oracle*)h;
  Level& L = O.lev.back();
  const int64_t n = L.n;
  const int m = restart;
  std::vector<double> r(n);
  residual(L, x, b, r.data());
  const double r0 = norm2(r);
  hist[0] = 1.0;
  if (r0 == 0.0) return 0;
  int it = 0;
  std::vector<std::vector<double>> V(m + 1, std::vector<double>(n)), Z(m, std::vector<double>(n));
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gam(m + 1), w(n);
  while (it < maxit) {
    residual(L, x, b, r.data());
    double beta = norm2(r);
    if (beta / r0 <= tol) return it;
    for (int64_t i = 0; i < n; ++i) V[0][i] = r[i] / beta;
    std::fill(gam.begin(), gam.end(), 0.0);
    gam[0] = beta;
    int j = 0;
    for (; j < m && it < maxit; ++j) {
      std::fill(Z[j].begin(), Z[j].end(), 0.0);
      vcycle(O, (int)O.lev.size() - 1, Z[j].data(), V[j].data(), nu1, nu2);
      // w = L z (Dirichlet rows of z are zero; identity rows give 0)
      for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = L.rp[i]; k < L.rp[i + 1]; ++k) s += L.va[k] * Z[j][L.ci[k]];
        w[i] = L.dir[i] ? 0.0 : s;
      }
      for (int i = 0; i <= j; ++i) {
        double hij = 0.0;
        for (int64_t q = 0; q < n; ++q) hij += w[q] * V[i][q];
        H[i * m + j] = hij;
        for (int64_t q = 0; q < n; ++q) w[q] -= hij * V[i][q];
      }
      const double hn = norm2(w);
      H[(j + 1) * m + j] = hn;
      for (int64_t q = 0; q < n; ++q) V[j + 1][q] = hn > 0 ? w[q] / hn : 0.0;
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
      hist[it] = std::fabs(gam[j + 1]) / r0;
      if (hist[it] <= tol) { ++j; break; }
    }
    // y = H^{-1} gamma (upper triangular j x j), x += Z y
    std::vector<double> y(j);
    for (int i = j - 1; i >= 0; --i) {
      double s = gam[i];
      for (int k = i + 1; k < j; ++k) s -= H[i * m + k] * y[k];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < j; ++i)
      for (int64_t q = 0; q < n; ++q) x[q] += y[i] * Z[i][q];
    if (hist[it] <= tol) {
      residual(L, x, b, r.data());
      hist[it] = norm2(r) / r0;
      if (hist[it] <= tol) return it;
    }
  }
  return -5;
}

// ---------------------------------------------------------------------------
// Learned damping (not in the paper, which allows a diagonal weighting per
// subdomain in Eq. 11): a per-subdomain weight omega_i predicted by a small
// MLP from local features, trained on line-search-optimal weights.
//
// Label of subdomain i for residual r, as a coordinate line search of the
// additive step: with c_i = Rt_i^T (L_i^{-1} R_i r) (its own restricted
// correction at weight 1) and the whole RAV step s = sum_j omega_j c_j, the
// weight of subdomain i alone that minimises ||r - L (s + (w - omega_i) c_i)||_2
// is omega*_i = omega_i + <r', L c_i> / <L c_i, L c_i> with r' = r - L s,
// clipped to [0, 1.5] (omega_i when L c_i = 0).  Norms over free rows; L c_i is
// formed with the full sparse L.  omega: current weights (null: `fallback`).
// Features of the learned per-subdomain damping (not in the paper; they
// describe what the local system of subdomain i sees), 8 per subdomain p of
// level l, written to out[8 p + k]:
//   0  log10(eta_max / eta_min) over the 3^d Gauss points of the cells around vertex p
//   1  mean of log10 eta over those points
//   2  log10 of the largest cell aspect ratio (longest over shortest side) there
//   3  log10 of the smallest one
//   4  l / (levels - 1)  (0 for a single level)
//   5  (d * free box nodes + 1) / (d * box nodes + 1): the subdomain's size
//      over the box's (box nodes: 5^d on Q2-Q1, 3^d on Q1-Q1; free = inside
//      the domain and not on its boundary)
//   6  boundary box nodes / box nodes inside the domain
//   7  log10 of the mean cell diagonal around vertex p
void orc_patch_features(void* h, int l, double* out) {
  const Oracle& O = *(const Oracle*)h;
  const Level& L = O.lev[l];
  const int d = L.dim, nlev = (int)O.lev.size();
  for (int64_t p = 0; p < L.n_p; ++p) {
    int64_t v[3] = {0, 0, 0};
    vert_of(L, p, v);
    double emin = 1e300, emax = 0.0, lsum = 0.0, amax = 0.0, amin = 1e300, diag = 0.0;
    int nq = 0, ncell = 0;
    int64_t cl[3][2];
    int cnt[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) cnt[a] = cells_of_vertex(v[a], L.N, cl[a]);
    tensor_loop(d, cnt, [&](const int* k) {
      double lo[3] = {0, 0, 0}, hh[3] = {0, 0, 0}, hmax = 0.0, hmin = 1e300, d2 = 0.0;
      for (int a = 0; a < d; ++a) {
        lo[a] = L.xv[a][cl[a][k[a]]];
        hh[a] = L.xv[a][cl[a][k[a]] + 1] - lo[a];
        hmax = std::max(hmax, hh[a]);
        hmin = std::min(hmin, hh[a]);
        d2 += hh[a] * hh[a];
      }
      amax = std::max(amax, hmax / hmin);
      amin = std::min(amin, hmax / hmin);
      diag += std::sqrt(d2);
      ++ncell;
      int g3[3] = {3, 3, 3};
      tensor_loop(d, g3, [&](const int* t) {
        double x[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) x[a] = lo[a] + hh[a] * kGaussX[t[a]];
        const double eta = viscosity(O.P, x);
        emin = std::min(emin, eta);
        emax = std::max(emax, eta);
        lsum += std::log10(eta);
        ++nq;
      });
    });
    // box nodes J = q v - q + a, a = 0 .. 2q per axis
    int ext[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) ext[a] = 2 * L.q + 1;
    int nbox = 0, nin = 0, nbnd = 0, nfree = 0;
    tensor_loop(d, ext, [&](const int* a) {
      bool in = true, bnd = false;
      for (int ax = 0; ax < d; ++ax) {
        const int64_t J = L.q * v[ax] - L.q + a[ax];
        in = in && J >= 0 && J <= L.M - 1;
        bnd = bnd || J == 0 || J == L.M - 1;
      }
      ++nbox;
      nin += in;
      nbnd += in && bnd;
      nfree += in && !bnd;
    });
    double* f = out + 8 * p;
    f[0] = std::log10(emax / emin);
    f[1] = lsum / nq;
    f[2] = std::log10(amax);
    f[3] = std::log10(amin);
    f[4] = nlev > 1 ? (double)l / (double)(nlev - 1) : 0.0;
    f[5] = (double)(d * nfree + 1) / (double)(d * nbox + 1);
    f[6] = nin ? (double)nbnd / (double)nin : 0.0;
    f[7] = std::log10(diag / ncell);
  }
}

void orc_labels(void* h, int l, const double* r, const double* omega, double fallback, double* out) {
  const Level& L = ((Oracle*)h)->lev[l];
  const int64_t np = (int64_t)L.poff.size() - 1;
  std::vector<std::vector<double>> cs(np);
  std::vector<double> s(L.n, 0.0), rp(L.n, 0.0);
  for (int64_t p = 0; p < np; ++p) {
    const int64_t b0 = L.poff[p], ni = L.poff[p + 1] - b0;
    std::vector<double> rows;
    inverse_rows(L, p, false, rows);
    cs[p].resize(L.owned[p].size());
    for (size_t j = 0; j < L.owned[p].size(); ++j) {
      double v = 0.0;
      for (int64_t k = 0; k < ni; ++k) v += rows[j * ni + k] * r[L.pdof[b0 + k]];
      cs[p][j] = v;
      s[L.pdof[b0 + L.owned[p][j]]] += (omega ? omega[p] : fallback) * v;
    }
  }
  for (int64_t m = 0; m < L.n; ++m) {
    if (L.dir[m]) continue;
    double t = 0.0;
    for (int64_t k = L.rp[m]; k < L.rp[m + 1]; ++k) t += L.va[k] * s[L.ci[k]];
    rp[m] = r[m] - t;
  }
  std::vector<double> c(L.n, 0.0);
  for (int64_t p = 0; p < np; ++p) {
    const int64_t b0 = L.poff[p];
    for (size_t j = 0; j < L.owned[p].size(); ++j) c[L.pdof[b0 + L.owned[p][j]]] = cs[p][j];
    double num = 0.0, den = 0.0;
    for (int64_t m = 0; m < L.n; ++m) {
      if (L.dir[m]) continue;
      double t = 0.0;
      for (int64_t k = L.rp[m]; k < L.rp[m + 1]; ++k) t += L.va[k] * c[L.ci[k]];
      num += rp[m] * t;
      den += t * t;
    }
    const double base = omega ? omega[p] : fallback;
    double w = den > 0.0 ? base + num / den : base;
    out[p] = w < 0.0 ? 0.0 : (w > 1.5 ? 1.5 : w);
    for (size_t j = 0; j < L.owned[p].size(); ++j) c[L.pdof[b0 + L.owned[p][j]]] = 0.0;
  }
}

// MLP 8 -> 64 -> 64 -> 1 (ReLU, ReLU, omega = 1.5 sigmoid(z)).  Parameters in
// one vector: W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3.
static const int kH = 64, kF = 8;
static const int64_t kNParam = kH * kF + kH + kH * kH + kH + kH + 1;

void mlp_one(const double* P, const double* f, double* a1, double* a2, double* z) {
  const double *W1 = P, *b1 = W1 + kH * kF, *W2 = b1 + kH, *b2 = W2 + kH * kH, *W3 = b2 + kH, *b3 = W3 + kH;
  for (int i = 0; i < kH; ++i) {
    double s = b1[i];
    for (int k = 0; k < kF; ++k) s += W1[i * kF + k] * f[k];
    a1[i] = s > 0.0 ? s : 0.0;
  }
  for (int i = 0; i < kH; ++i) {
    double s = b2[i];
    for (int k = 0; k < kH; ++k) s += W2[i * kH + k] * a1[k];
    a2[i] = s > 0.0 ? s : 0.0;
  }
  double s = b3[0];
  for (int k = 0; k < kH; ++k) s += W3[k] * a2[k];
  *z = s;
}

long long orc_mlp_nparam() { return kNParam; }

void orc_mlp_forward(const double* P, const double* X, long long n, double* out) {
  double a1[kH], a2[kH], z;
  for (long long s = 0; s < n; ++s) {
    mlp_one(P, X + s * kF, a1, a2, &z);
    out[s] = 1.5 / (1.0 + std::exp(-z));
  }
}

// Mean squared error (1/n) sum_s (omega_s - y_s)^2 and its gradient with
// respect to every parameter (backpropagation through the three layers).
double orc_mlp_loss_grad(const double* P, const double* X, const double* y, long long n, double* grad) {
  const double *W2 = P + kH * kF + kH, *W3 = W2 + kH * kH + kH;
  double *gW1 = grad, *gb1 = gW1 + kH * kF, *gW2 = gb1 + kH, *gb2 = gW2 + kH * kH, *gW3 = gb2 + kH,
         *gb3 = gW3 + kH;
  std::fill(grad, grad + kNParam, 0.0);
  double loss = 0.0, a1[kH], a2[kH], z, d2[kH], d1[kH];
  for (long long s = 0; s < n; ++s) {
    const double* f = X + s * kF;
    mlp_one(P, f, a1, a2, &z);
    const double sg = 1.0 / (1.0 + std::exp(-z));
    const double om = 1.5 * sg;
    const double e = om - y[s];
    loss += e * e / n;
    const double dz = 2.0 * e / n * 1.5 * sg * (1.0 - sg);
    gb3[0] += dz;
    for (int k = 0; k < kH; ++k) {
      gW3[k] += dz * a2[k];
      d2[k] = a2[k] > 0.0 ? dz * W3[k] : 0.0;
    }
    for (int i = 0; i < kH; ++i) {
      gb2[i] += d2[i];
      for (int k = 0; k < kH; ++k) gW2[i * kH + k] += d2[i] * a1[k];
    }
    for (int k = 0; k < kH; ++k) {
      double s2 = 0.0;
      for (int i = 0; i < kH; ++i) s2 += W2[i * kH + k] * d2[i];
      d1[k] = a1[k] > 0.0 ? s2 : 0.0;
    }
    for (int i = 0; i < kH; ++i) {
      gb1[i] += d1[i];
      for (int k = 0; k < kF; ++k) gW1[i * kF + k] += d1[i] * f[k];
    }
  }
  return loss;
}

// Rounds v[i] to the given format (prec 1 fp32, 2 bf16, 3 fp8 e4m3), for tests.
void orc_round_format(int prec, const double* v, double* out, long long n) {
  for (long long i = 0; i < n; ++i) out[i] = fmt_round(prec, v[i]);
}

}  // extern "C"
