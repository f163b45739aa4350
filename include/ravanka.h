/*
 * ravanka.h -- C ABI of the GB300 restricted additive Vanka multigrid library.
 *
 * Method: Saberi, Meschke, Vogel, "A restricted additive Vanka smoother for
 * geometric multigrid".  The library solves the Stokes saddle-point system
 * L x = b, L = [A B; B^T C] (Sec. 2, Eqs. 5-7 and 9) discretised with
 * inf-sup-stable Q2-Q1 (Taylor-Hood) elements (C = 0, Sec. 2 after Eq. 7), or
 * with the paper's own equal-order Q1-Q1 pair and the pressure stabilisation
 * C = -beta sum_e h_e^2 (grad q, grad p)_e of Eq. 8, on tensor-product box
 * grids, by a geometric multigrid V-cycle (Sec. 2, Fig. 1) whose smoother is
 * one of
 *   RAV  restricted additive Vanka, Eq. 13 (the method of the paper),
 *   AV   additive Vanka, Eq. 12,
 *   MV   multiplicative Vanka, Eq. 11, run in a 4^d-coloured patch order,
 * each applied as x <- x + S (b - L x) (Eq. 10).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Numbering (all DoFs, Dirichlet ones included, live in x):
 *      Q2 node I in [0,2N]^d, node id = I0 + (2N+1)(I1 + (2N+1) I2),
 *      velocity DoF = d*id + c (components interleaved per node),
 *      pressure vertex v in [0,N]^d, id = v0 + (N+1)(v1 + (N+1) v2),
 *      pressure DoF = n_u + id, n_u = d (2N+1)^d, n = n_u + (N+1)^d.
 *    On Q1-Q1 the velocity nodes are the vertices: node id = vertex id,
 *      n_u = d (N+1)^d.
 *  * Every boundary velocity node is a Dirichlet node for all components.  Its row
 *    of L is the identity row; the residual is defined as 0 there; the
 *    Dirichlet value lives in x (no lifting).
 *  * Level 0 is the coarsest, level n_levels-1 the finest (N cells per axis);
 *    level l has N / 2^(n_levels-1-l) cells per axis.
 *  * Pointers named *_dev are CUDA device pointers owned by the caller;
 *    pointers named *_host are host pointers owned by the caller.  The
 *    library never frees caller memory.  Library objects (matrices, patch
 *    inverses, work vectors, the coarse inverse) are owned by the handle and
 *    released by mg_destroy / vanka_destroy.
 *  * stream is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *    work on it and return without synchronising, except where stated.
 *  * Every call returns RAV_OK (0) or a negative RAV_ERR_* code; nothing
 *    aborts and no device code traps.  rav_strerror() names a code.
 */
#ifndef RAVANKA_H
#define RAVANKA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rav_mg rav_mg;             /* grid hierarchy + assembled operators */
typedef struct rav_smoother rav_smoother; /* Vanka subdomains + stored inverses   */
typedef void* rav_stream;                 /* cudaStream_t                         */

enum {
  RAV_OK = 0,
  RAV_ERR_ARG = -1,             /* invalid argument or size                    */
  RAV_ERR_CUDA = -2,            /* a CUDA runtime call failed                  */
  RAV_ERR_SINGULAR_PATCH = -3,  /* a local system L_i could not be factorised  */
  RAV_ERR_SINGULAR_COARSE = -4, /* the bordered coarse system is singular      */
  RAV_ERR_NOT_CONVERGED = -5,   /* maxit reached before the tolerance          */
  RAV_ERR_DIVERGED = -6,        /* residual grew beyond the divergence guard   */
  RAV_ERR_NAN = -7,             /* non-finite residual                         */
  RAV_ERR_TIMEOUT = -8          /* a bounded device wait gave up               */
};

enum rav_bc { RAV_BC_CAVITY = 0, RAV_BC_NOSLIP = 1, RAV_BC_QUADRATIC = 2 };
/* Discretisation: Taylor-Hood Q2-Q1 (C = 0), or equal-order Q1-Q1 with the
 * pressure stabilisation of Eq. 8. */
enum rav_element { RAV_ELEM_Q2Q1 = 0, RAV_ELEM_Q1Q1 = 1 };
enum rav_forcing { RAV_F_NONE = 0, RAV_F_PSI = 1, RAV_F_SINKER = 2, RAV_F_QUADRATIC = 3 };
enum rav_smoother_kind { RAV_RAV = 0, RAV_AV = 1, RAV_MV_COLOURED = 3 };
/* Storage of the RAV inverse rows.  RAV_F64: fp64, factored through the block
 * form of L_i^{-1} (rows of K_i^{-1} of the owned nodes, w = A_i^{-1} b and
 * 1/s; see vanka_setup).  RAV_F64_ROWS: the owned rows of L_i^{-1} themselves
 * in fp64 (the storage of Sec. 4.3 as written).  RAV_F32 / RAV_BF16 / RAV_FP8:
 * the owned rows rounded to nearest-even into that format (fp8 e4m3 with an
 * fp32 scale max|row|/448 per row), applied with fp32 accumulation.
 * RAV_F32_FACT / RAV_BF16_FACT: the factored storage of RAV_F64 with every
 * stored value (K_i^{-1} rows, w, 1/s) rounded to nearest-even into fp32 /
 * bf16, applied with fp32 accumulation (the correction is added to x in fp64).
 * AV and MV store all rows in fp64 (RAV_F64 or RAV_F64_ROWS). */
enum rav_precision {
  RAV_F64 = 0,
  RAV_F32 = 1,
  RAV_BF16 = 2,
  RAV_FP8 = 3,
  RAV_F64_ROWS = 4,
  RAV_F32_FACT = 5,
  RAV_BF16_FACT = 6
};

/* Problem on the unit square (dim 2) or cube (dim 3).
 *  coords_host: dim*(N+1) finest-level vertex coordinates, axis-major, strictly
 *               increasing, or NULL for a uniform grid.  Coarser levels use
 *               every 2nd, 4th, ... vertex.
 *  viscosity:   eta(x) = eta0 * 10^(max_k s_k exp(-|x - c_k|^2 / (2 rho_k^2)))
 *               with blobs_host = nblobs * (cx, cy, cz, rho, s); eta0 if nblobs = 0.
 *  bc:          RAV_BC_CAVITY (u = e_0 on the face x_{d-1} = 1, edges and corners
 *               of that face included, 0 elsewhere), RAV_BC_NOSLIP (u = 0),
 *               RAV_BC_QUADRATIC (u = (y^2, x^2) in 2-D, (y^2, z^2, x^2) in 3-D).
 *  element:     rav_element (zero-initialised structs get Q2-Q1).
 *  beta:        the constant of Eq. 8 (Q1-Q1 only; finite, >= 0; h_e is the
 *               cell diameter).  Ignored for Q2-Q1. */
typedef struct rav_problem {
  int dim;
  int N;
  const double* coords_host;
  double eta0;
  int nblobs;
  const double* blobs_host;
  int bc;
  int element;
  double beta;
} rav_problem;

/* Builds the hierarchy: per level the operator of Eq. 7 (Q2-Q1, or Q1-Q1 with
 * the C of Eq. 8) assembled from 3^d-point Gauss quadrature (the paper
 * assembles on every grid, Sec. 4), the interpolation tables of the nested
 * velocity (Q2 or Q1) and Q1 pressure spaces, and on level 0 the explicit
 * inverse of the bordered system [L e_p; e_p^T 0] for the LU coarse solve of
 * Sec. 2.  Requires N divisible by 2^(n_levels-1) and a coarsest grid of at
 * least 2 cells per axis.  Synchronises the stream before returning.
 * Errors: RAV_ERR_ARG, RAV_ERR_CUDA, RAV_ERR_SINGULAR_COARSE. */
int mg_setup(const rav_problem* p, int n_levels, rav_stream stream, rav_mg** out);
void mg_destroy(rav_mg* mg);

/* Sizes of level l: out[0] = n_u, out[1] = n_p, out[2] = n, out[3] = nnz of L,
 * out[4] = N (cells per axis). */
int rav_get_counts(const rav_mg* mg, int level, int64_t out[5]);

/* Copies the CSR form of level l's operator into caller device buffers:
 * rowptr_dev[n+1] (int64), col_dev[nnz] (int32, ascending per row),
 * val_dev[nnz] (fp64).  Structural entries that cancel are kept. */
int rav_get_csr(const rav_mg* mg, int level, int64_t* rowptr_dev, int32_t* col_dev, double* val_dev,
                rav_stream stream);

/* Finest-level right-hand side: b_u = int v . f over 3^d Gauss points of every
 * cell, b_p = 0 (Eq. 6), b = Dirichlet value on Dirichlet rows.  forcing is one
 * of rav_forcing (PSI: manufactured curl of sin^2(pi x) sin^2(pi y) with
 * p = cos(pi x) cos(pi y); SINKER: f = (0,..,0,-max_k exp(-|x-c_k|^2/(2 rho_k^2)));
 * QUADRATIC: the body force of the quadratic exact solution). b_dev has n entries. */
int rav_assemble_rhs(rav_mg* mg, int forcing, double* b_dev, rav_stream stream);

/* x_dev[n] = Dirichlet values on Dirichlet DoFs, 0 elsewhere (the initial guess). */
int rav_initial_guess(rav_mg* mg, double* x_dev, rav_stream stream);

/* r = b - L x on free rows, r = 0 on Dirichlet rows (the residual of Eq. 10), on
 * level l; all three vectors have that level's n entries.  If norm_host is not
 * NULL the call synchronises and stores ||r||_2 there.  Every residual of the
 * library reads a sliced-ELL copy of L that leaves out entries of magnitude at
 * most 2^-46 of the largest in their row: on these grids those are the
 * quadrature roundoff of couplings that cancel exactly (a quarter of the
 * stored entries, within a few ulps of zero), genuine couplings staying above
 * 1e-7 of their row; the effect on r is below the rounding of its fp64 sums.
 * rav_get_csr returns L as assembled, those entries included. */
int rav_residual(rav_mg* mg, int level, const double* x_dev, const double* b_dev, double* r_dev,
                 double* norm_host, rav_stream stream);

/* Launch shape of the residual on level l (every residual of the library
 * except rav_residual_norm_noalloc, which always uses 1): threads_per_row
 * threads (1, 2, 4, 8, 16 or 32) share each row and add their partial sums by
 * shuffles.  mg_setup times every choice on every level (5 launches each on
 * the level's work vectors) and keeps the fewest threads within 3 % of the
 * fastest, so the choice can differ between runs where two are that close.  The
 * result differs only in the order of the fp64 additions.  Setting it waits
 * for the device and drops the captured V-cycle graphs (recaptured on next
 * use).  RAV_ERR_ARG for another value or level.  rav_get_residual_split
 * returns the current value (or RAV_ERR_ARG). */
int rav_set_residual_split(rav_mg* mg, int level, int threads_per_row);
int rav_get_residual_split(const rav_mg* mg, int level);

/* Node-blocked residual on level l (Q2-Q1 hierarchies): the gradient form of
 * Eq. 7 gives the d velocity rows of a node the same velocity columns and
 * values (A = I_d (x) K), so one thread per velocity node reads each stored K
 * entry once for the d components (x as a d-vector) and each pressure column
 * once with the node's d entries of B; pressure rows keep a row-wise copy of
 * their own.  Same fp64 products as the row-wise residual, about 40 % (2-D)
 * or 60 % (3-D) fewer stored bytes; results differ in the order of the
 * additions.  mg_setup times it against the row-wise kernel on every level and
 * keeps it where 3 % faster (only then does it hold its memory).  Used when x
 * is 16-byte aligned (the row-wise kernel serves other x).  enable = 0 frees it.
 * Synchronises the stream and drops the captured V-cycle graphs.  RAV_ERR_ARG
 * on Q1-Q1 levels or when a level's component rows differ.
 * rav_get_residual_blocked returns 1 or 0 (or RAV_ERR_ARG). */
int rav_set_residual_blocked(rav_mg* mg, int level, int enable, rav_stream stream);
int rav_get_residual_blocked(const rav_mg* mg, int level);

/* FP32 residuals on the levels between the coarsest and the finest that hold
 * at least min_dofs DoFs (enable = 1; 0 returns to fp64 everywhere; smaller
 * levels are latency-bound and keep fp64): r = b - L x (Eq. 10) there with the operator values
 * rounded to fp32, x rounded to fp32 before each residual (one conversion
 * kernel), products summed in fp32 and r = b - sum formed in fp64.  The finest
 * level's residual, which measures convergence and feeds the outer loop, and
 * the coarse solve stay fp64.  On the levels in between r then
 * carries fp32 rounding (about 2^-24 of sum_k |a_k x_k| per row), which the
 * coarse-grid correction tolerates like the reduced-precision subdomain
 * inverses.  Allocates an fp32 copy of each such level's operator and of its
 * x, synchronises the stream and drops the captured cycles of every smoother
 * of mg.  RAV_ERR_ARG for other values or a negative min_dofs.
 * rav_get_coarse_residual_f32 returns
 * 1 when it is on, 0 when off.  The paper has no counterpart. */
int rav_set_coarse_residual_f32(rav_mg* mg, int enable, int64_t min_dofs, rav_stream stream);
int rav_get_coarse_residual_f32(const rav_mg* mg);

/* FP32 grid transfers in the V-cycle (Q2-Q1; enable = 1; 0 returns to fp64):
 * the restriction of each level's residual (rounded to fp32 by the residual
 * kernel) and the prolongation of each coarse correction (x rounded to fp32
 * by one conversion kernel) use the interpolation weights in fp32 and fp32
 * sums; b of the coarser level and the update of x are fp64 (Sec. 2's
 * transfers, computed to fp32 rounding, about 2^-24 of the sum of |terms| per
 * entry).  rav_restrict and rav_prolong_add stay fp64.  Allocates fp32 copies
 * of the weight tables and one fp32 vector per level, synchronises the stream
 * and drops the captured cycles of every smoother of mg.  RAV_ERR_ARG for
 * other values or a Q1-Q1 hierarchy.  rav_get_transfers_f32 returns 1 when it
 * is on, 0 when off.  The paper has no counterpart. */
int rav_set_transfers_f32(rav_mg* mg, int enable, rav_stream stream);
int rav_get_transfers_f32(const rav_mg* mg);

/* Same residual r = b - L x on level l as rav_residual, plus ||r||_2 written to
 * the caller's device scalar norm_dev, with no memory allocation of any kind
 * and no host synchronisation.  The paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc at the point where they need the
 * residual (for instance while their stream is being captured into a CUDA
 * graph, or in a loop that may only use memory reserved beforehand).
 *  * Scratch: the norm's partial sums (one per 256 rows) go to a fixed array of
 *    16,384 doubles (128 KiB) that the library keeps in device memory; every
 *    GPU that loads the library holds it until the process exits.  A level
 *    with more than 4,194,304 row slots (rows padded to slices of 32; 2-D
 *    grids above about 680 x 680 cells, 3-D above about 55^3) is rejected with
 *    RAV_ERR_ARG before anything is launched.
 *  * The first call on a device looks up that array's device address (with
 *    the device current) and caches it; make that first call before any
 *    stream capture.  Call with the device of mg (the one current at
 *    mg_setup) current: any other current device gives RAV_ERR_ARG before
 *    anything is launched.
 *  * All calls share the array and it keeps the last call's contents (every
 *    call overwrites the entries it uses, nothing needs clearing first): calls
 *    whose kernels overlap on the GPU (different streams, no ordering) race
 *    and may return wrong norms.  r_dev and norm_dev belong to the caller. */
int rav_residual_norm_noalloc(rav_mg* mg, int level, const double* x_dev, const double* b_dev, double* r_dev,
                              double* norm_dev, rav_stream stream);

/* Grid transfers between level l-1 (coarse) and l (fine), canonical nested
 * interpolation P of the velocity (Q2 or Q1) and Q1 pressure spaces (the paper builds
 * its transfers from the grid hierarchy, Sec. 2):
 *   rav_restrict:   bc = P^T rf, then 0 on coarse Dirichlet rows;
 *   rav_prolong_add: xf += P xc on free fine DoFs (fine Dirichlet DoFs untouched). */
int rav_restrict(rav_mg* mg, int level, const double* rf_dev, double* bc_dev, rav_stream stream);
int rav_prolong_add(rav_mg* mg, int level, const double* xc_dev, double* xf_dev, rav_stream stream);

/* Coarse solve on level 0 (Sec. 2, LU to machine accuracy): x = first n_0
 * entries of [L e_p; e_p^T 0]^{-1} [b masked to free rows; 0]; the pressure of
 * x has zero sum. */
int rav_coarse_solve(rav_mg* mg, const double* b_dev, double* x_dev, rav_stream stream);

/* Builds the Vanka subdomains of every level above the coarsest (Sec. 3):
 * subdomain i = pressure DoF p_i plus every free velocity DoF of the cells
 * around vertex i.  Factorises each local system L_i = R_i L R_i^T in fp64 and
 * stores
 *   RAV: the rows of L_i^{-1} of the DoFs owned by i (Sec. 4.3), ownership =
 *        vertex floor(I/2) for a velocity DoF at Q2 node I, own vertex for p_i;
 *   AV, MV: all rows of L_i^{-1}.
 * precision is one of rav_precision: the rows themselves (RAV_F64_ROWS, or
 * rounded into fp32 / bf16 / fp8 e4m3 with an fp32 scale per row), or the
 * factored form of the block inverse (RAV_F64, RAV_F32_FACT, RAV_BF16_FACT);
 * reduced formats are applied with fp32 accumulation (RAV only; AV and MV
 * take RAV_F64 or RAV_F64_ROWS, both meaning fp64 full inverses).  omega is
 * the damping of every subdomain (Eq. 11).  Also times the launch shapes of
 * the factored apply (rav_set_apply_split).  Synchronises the stream.
 * On a Q1-Q1 hierarchy subdomain i holds p_i and the free velocity DoFs of the
 * 3^d vertices around vertex i and owns exactly the velocity DoFs of vertex i
 * and p_i (the paper's restricted set, Sec. 3); RAV takes every storage
 * (factored with s = c_ii - b^T A^{-1} b, c_ii the stabilisation's diagonal
 * entry, or the d + 1 owned rows over the 3^d d + 1 box positions), one thread
 * per subdomain and no apply split; AV and MV store the full fp64 L_i^{-1}
 * over the box positions.
 * Errors: RAV_ERR_ARG, RAV_ERR_CUDA, RAV_ERR_SINGULAR_PATCH. */
int vanka_setup(rav_mg* mg, int kind, int precision, double omega, rav_stream stream, rav_smoother** out);
void vanka_destroy(rav_smoother* sm);

/* Launch shape of the factored RAV apply (RAV_F64, RAV_F32_FACT,
 * RAV_BF16_FACT) on level l: split threads per owned node (1, 2, 4 or 8 in
 * 2-D; 1, 2 or 4 in 3-D) share the sum over the subdomain's box nodes and add
 * their partial sums by shuffles.  vanka_setup times every choice on every
 * level (5 applies each) and keeps the fewest threads within 3 % of the
 * fastest.  The stored K_i^{-1} rows are grouped by 32/split
 * subdomain nodes, so setting it regroups them on the device (synchronises
 * the stream, allocates and frees one copy) and drops the captured V-cycle
 * graphs of this smoother.  Results differ only in the order of additions.
 * RAV_ERR_ARG for other values, levels or storage (on Q1-Q1 only 1 is
 * accepted).  rav_get_apply_split returns the current value (or RAV_ERR_ARG). */
int rav_set_apply_split(rav_smoother* sm, int level, int split, rav_stream stream);
int rav_get_apply_split(const rav_smoother* sm, int level);

/* Staged apply of the reduced factored storage (RAV_F32_FACT, RAV_BF16_FACT;
 * Q2-Q1) on level l: the same Eq. 13 step computed by thread blocks that
 * each copy the fp32 residual of their tile of subdomain boxes (tiles of
 * vertices, chosen per level) into shared memory once, then stream the stored
 * values of their subdomains in per-thread chunks (the 2^d owned rows of
 * K_i^{-1} and w at one box node) with threads_per_subdomain threads per
 * subdomain: 1 (tiles of fixed shape, 16 x 24 vertices in 2-D with each
 * thread taking three subdomains in turn, 3 x 3 x 3 in 3-D; box offsets known
 * at compile time, the stream kept in flight in registers), 2 (2-D and 3-D)
 * or 4 (3-D), the partial sums of several threads meeting by shuffles.  0
 * returns to the grouped kernel of rav_set_apply_split.  The chunks are a
 * second copy of the stored values, built from the grouped storage (same
 * rounded values) when set, for 2 and 4 with the tiling ranked first for that
 * thread count (fewest idle thread slots, best use of the last wave, least
 * halo); vanka_setup times the grouped kernel and the staged one (1 thread;
 * the three best-ranked tilings of 2 and 4 threads) on every level and keeps
 * the staged one where it is 3 % faster.  Setting it synchronises the
 * stream and drops this smoother's captured cycles.  Results differ from the
 * grouped kernel only in the order of the fp32 additions.  RAV_ERR_ARG for
 * other values or storage (0 is accepted everywhere).  rav_get_apply_staged
 * returns the current value (or RAV_ERR_ARG). */
int rav_set_apply_staged(rav_smoother* sm, int level, int threads_per_subdomain, rav_stream stream);
int rav_get_apply_staged(const rav_smoother* sm, int level);

/* Fused smoothing (RAV only; on Q1-Q1 with RAV_F64 storage, on Q2-Q1 with
 * the factored storages RAV_F64, RAV_F32_FACT, RAV_BF16_FACT; RAV_ERR_ARG
 * otherwise): with enable != 0 every smoothing step of this smoother runs as
 * one kernel that computes the residual of Eq. 10 on each tile's subdomain
 * boxes (Q1-Q1: tiles of 16 x 16 or 8 x 8 x 4 vertices plus a one-vertex
 * halo; Q2-Q1: tiles of 16 x 16 or 8 x 8 x 4 vertices, their boxes reaching
 * two Q2 nodes past the tile, kept in shared memory in the accumulation type
 * of the storage) and applies the subdomain corrections of Eq. 13, reading
 * one iterate buffer and writing another (the library allocates the second
 * one per level); 0 returns to the residual + apply kernels.  On Q2-Q1 the
 * stored rows are regrouped for one thread per owned node (as
 * rav_set_apply_split(sm, l, 1)).  Results agree with the two-kernel path to
 * rounding (the fused residual sums the rows in the order of the residual
 * kernel with one thread per row).  Synchronises the device and drops this
 * smoother's captured cycles. */
int rav_set_fused_smoothing(rav_smoother* sm, int enable);

/* Replaces the damping of level l's subdomains by w_dev[n_p(l)] (fp32, device),
 * e.g. the per-subdomain weights of a learned model. */
int rav_set_patch_omega(rav_smoother* sm, int level, const float* w_dev, rav_stream stream);

/* Subdomain structure of level l for inspection: counts_out[0] = number of
 * subdomains, counts_out[1] = total DoFs over all subdomains. */
int rav_get_patch_counts(const rav_smoother* sm, int level, int64_t counts_out[2]);
/* offsets_dev[np+1], dofs_dev[total] (each list ascending), owner_dev[n]
 * (owning subdomain per DoF, -1 for Dirichlet DoFs); int32, device. */
int rav_get_patches(const rav_smoother* sm, int level, int32_t* offsets_dev, int32_t* dofs_dev,
                    int32_t* owner_dev, rav_stream stream);
/* Stored inverse rows of subdomains [first, first+count) of level l, expanded
 * to fp64 (scale applied) in the sorted DoF order of each subdomain, into
 * out_dev[count][rows_max][cols_max] (zero padded); rows_max/cols_max are
 * 2^d d + 1 and 5^d d + 1 for RAV, 5^d d + 1 for both otherwise; on a Q1-Q1
 * hierarchy d + 1 and 3^d d + 1 for RAV, 3^d d + 1 for both otherwise. */
int rav_get_inverse_rows(const rav_smoother* sm, int level, int64_t first, int64_t count, double* out_dev,
                         rav_stream stream);

/* steps smoothing steps x <- x + S (b - L x) on level l (Eq. 10 with S from
 * Eq. 13, 12 or 11).  x_dev, b_dev have n(l) entries. */
int vanka_smooth(rav_smoother* sm, int level, double* x_dev, const double* b_dev, int steps, rav_stream stream);

/* The subdomain part of one RAV or AV step on level l (Eq. 13 or 12 applied to a
 * given residual): x += S r, with r_dev the residual of that level (zero on
 * Dirichlet rows, e.g. from rav_residual).  vanka_smooth = rav_residual +
 * vanka_apply.  RAV_ERR_ARG for MV, whose residual changes inside the sweep. */
int vanka_apply(rav_smoother* sm, int level, const double* r_dev, double* x_dev, rav_stream stream);

/* One V(nu_pre, nu_post) cycle on the finest level (Sec. 2, Fig. 1): smoothing,
 * residual restriction, recursive coarse correction with x_c = 0, the coarse
 * solve on level 0, prolongation, smoothing.  x_dev is updated in place.
 * By default the cycle's kernels are captured into a CUDA graph on the first
 * call for a given (sm, x_dev, b_dev, nu_pre, nu_post) and replayed on stream
 * afterwards (the first call therefore must not happen during a capture of
 * stream by the caller); the graph reads x_dev, b_dev and the smoother's
 * damping at replay time.  While the timing hook records, cycles are
 * launched kernel by kernel. */
int vcycle(rav_mg* mg, rav_smoother* sm, double* x_dev, const double* b_dev, int nu_pre, int nu_post,
           rav_stream stream);

/* Turns the graph replay of vcycle / solve on (default) or off (kernel-by-kernel
 * launches; frees the captured graphs). */
int rav_set_graphs(rav_mg* mg, int enable);

typedef struct rav_solve_opts {
  double tol;      /* stop when ||r_k||_2 / ||r_0||_2 <= tol (Sec. 4 uses 1e-8) */
  int maxit;       /* V-cycles (stationary) or inner iterations (FGMRES)         */
  int nu_pre, nu_post;
  int outer;       /* 0 stationary multigrid, 1 FGMRES(restart) with one V-cycle as
                      right preconditioner                                         */
  int restart;     /* FGMRES restart length (30)                                */
  double diverge;  /* stop with RAV_ERR_DIVERGED when the ratio exceeds this     */
  double fallback_rho; /* stationary only, > 0: after a V-cycle that reduced the
                          residual by a factor worse than this, reset every
                          subdomain's damping to the fixed value of vanka_setup
                          (once) and go on; 0 disables                      */
} rav_solve_opts;

typedef struct rav_solve_info {
  int iterations;         /* V-cycles or FGMRES inner iterations done           */
  int status;             /* RAV_OK or the error returned                       */
  double final_ratio;     /* ||r||/||r_0|| at exit                              */
  double* history_host;   /* optional, maxit+1 entries: ratio after each step  */
  int fell_back;          /* 1 if the fallback to fixed damping happened        */
} rav_solve_info;

/* Solves L x = b from the given x (usually rav_initial_guess).  Host-driven:
 * synchronises once per V-cycle (stationary) or inner iteration (FGMRES) to
 * read the residual norm.  Stationary: each V-cycle replays a graph and starts
 * from the residual just computed for the norm.  FGMRES (flexible GMRES, right
 * preconditioned by one V-cycle from a zero guess, restarted every `restart`
 * iterations) orthogonalises by classical Gram-Schmidt applied twice; the
 * least-squares update runs on the host.  The residual norm, the Krylov
 * vectors and the solution stay fp64 whatever the smoother's storage.
 * info may be NULL; otherwise it is filled on every return, failures included
 * (status = the returned code; iterations, final_ratio and history up to the
 * iteration reached; fell_back = 0 unless the stationary fallback happened). */
int solve(rav_mg* mg, rav_smoother* sm, double* x_dev, const double* b_dev, const rav_solve_opts* opts,
          rav_solve_info* info, rav_stream stream);

/* ---- Learned damping per subdomain ---------------------------------------
 * The paper allows a diagonal weighting omega_i per subdomain (Eq. 11) and
 * uses one constant.  These calls predict omega_i with an MLP 8 -> 64 -> 64 -> 1
 * (ReLU, ReLU, omega = 1.5 sigmoid(z)) from 8 features per subdomain, and
 * train it on line-search-optimal weights gathered from the method's own runs.
 * Parameters: 4801 fp32 values W1[64][8], b1[64], W2[64][64], b2[64], W3[64],
 * b3 (device).  Inference rounds the weights to fp16 and accumulates in fp32.
 *
 * rav_patch_features: feat_dev[n_p(l) * 8] (fp32) for level l: log10(eta_max /
 *   eta_min) and mean log10 eta over the Gauss points of the cells around the
 *   vertex, log10 of the largest and smallest cell aspect ratio there,
 *   l / (levels - 1), subdomain DoFs / box positions, fraction of in-domain box
 *   nodes on the Dirichlet boundary, log10 of the mean cell diagonal.
 * rav_label_collection(sm, 1): clears and starts accumulating, in every RAV
 *   smoothing step (vanka_smooth, vcycle, solve; V-cycles then run kernel by
 *   kernel), the coordinate line-search weight of each subdomain:
 *   omega*_i = clip(omega_i + <r', L c_i> / <L c_i, L c_i>, 0, 1.5), where r is
 *   the step's residual, c_i the subdomain's own restricted correction with
 *   weight 1, s = sum_j omega_j c_j the whole step and r' = r - L s: the exact
 *   minimiser over w of ||r - L (s + (w - omega_i) c_i)||_2.  (sm, 0) stops.
 * rav_read_labels: label_dev[n_p(l)] = mean omega*_i (the fixed damping where
 *   no sample was taken).
 * rav_mlp_forward: omega_dev[n] for feature rows X_dev[n * 8].
 * rav_mlp_loss_grad: mean squared error of omega against y_dev and its
 *   gradient grad_dev[4801] (fp32, deterministic); work_dev must hold
 *   ceil(n / 64) * 4802 floats.  loss_dev may be NULL.
 * rav_adam_step: one Adam update (beta 0.9 / 0.999, eps 1e-8) of params_dev
 *   with moments m_dev, v_dev; t = 1, 2, ... the step number.
 * rav_set_learned_omega: features -> MLP -> omega_i on every level of sm, then
 *   omega_i <- m + shrink (omega_i - m) with m the level's mean prediction
 *   (shrink in [0, 1]: 1 keeps the per-subdomain predictions, 0 gives one
 *   predicted weight per level); replaces the damping, rav_reset_omega
 *   restores the fixed value. */
int rav_mlp_nparam(void);
int rav_patch_features(rav_smoother* sm, int level, float* feat_dev, rav_stream stream);
int rav_label_collection(rav_smoother* sm, int enable);
int rav_read_labels(rav_smoother* sm, int level, float* label_dev, rav_stream stream);
int rav_mlp_forward(const float* params_dev, const float* X_dev, int64_t n, float* omega_dev, rav_stream stream);
int rav_mlp_loss_grad(const float* params_dev, const float* X_dev, const float* y_dev, int64_t n, float* grad_dev,
                      float* loss_dev, float* work_dev, int64_t work_floats, rav_stream stream);
int rav_adam_step(float* params_dev, float* m_dev, float* v_dev, const float* grad_dev, float lr, int t,
                  rav_stream stream);
int rav_set_learned_omega(rav_smoother* sm, const float* params_dev, double shrink, rav_stream stream);
int rav_reset_omega(rav_smoother* sm, rav_stream stream);

/* ---- Batched solves: many problems x several right-hand sides ------------
 * A batch groups nprob hierarchies (any mix of sizes and depths, one
 * dimension, one element: Q2-Q1 or Q1-Q1) with their RAV smoothers, which must store dense owned rows
 * (RAV_F32 or RAV_F64_ROWS), and advances nrhs (1, 2, 4 or 8) right-hand
 * sides of every problem together.  Vectors of problem p are RHS-interleaved:
 * x_dev[p][row * nrhs + k], n(p) * nrhs doubles, numbering as above; with
 * nrhs >= 2 they must be 16-byte aligned (rows are read two doubles at a
 * time), else batch_vcycle and solve_batched return RAV_ERR_ARG.  Each
 * phase of the V-cycle is one kernel launch over all problems; the cycle is
 * captured into a CUDA graph on first use and replayed.  Per right-hand side
 * the result equals the single-problem vcycle() with the same smoother bit for
 * bit when that hierarchy's residual uses one thread per row
 * (rav_set_residual_split(mg, l, 1) on every level).  batch_setup times candidate launch shapes on the batch's own data and
 * keeps the fastest (batch_get_tuning reports them).  The batch does not own
 * the hierarchies or smoothers; destroy it first. */
typedef struct rav_batch rav_batch;
int batch_setup(rav_mg* const* mgs, rav_smoother* const* sms, int nprob, int nrhs, rav_stream stream,
                rav_batch** out);
void batch_destroy(rav_batch* bt);
/* out[0] = threads per block of the residual kernel, out[1] = of the apply kernel. */
int batch_get_tuning(const rav_batch* bt, int out[2]);
/* The RAV apply of 2-D Q2-Q1 batches with FP32 rows and 8 right-hand sides
 * can run tiled: a block of 32 x ty vertices stages the FP32 residual of its
 * subdomain boxes (Sec. 3's restriction) in shared memory with coalesced
 * copies and adds the velocity corrections (Eq. 13) to x by contiguous rows of
 * owned nodes, with the same sums in the same order as the untiled kernel (bit
 * for bit the same results); split = 2 gives each row of vertices two warps,
 * owned rows 0-3 and 4-8 of the same subdomains.  batch_setup chooses per
 * depth between untiled and ty in {2, 4} x split in {1, 2} by timing each on
 * the batch's own data.
 * batch_set_apply_tile: ty = 2 or 4 tiles every depth with the given split, 0
 * none, -1 restores batch_setup's choice (split 1 or 2 is still required);
 * synchronises the stream and drops the captured cycle; RAV_ERR_ARG for other
 * values, or for ty 2 or 4 on any other batch.
 * batch_get_apply_tile: out[0] = ty in use at depth (0 = finest; 0 =
 * untiled), out[1] = split (1 when untiled); RAV_ERR_ARG outside 0 .. depths
 * - 1.  The paper has no counterpart. */
int batch_set_apply_tile(rav_batch* bt, int ty, int split, rav_stream stream);
int batch_get_apply_tile(const rav_batch* bt, int depth, int out[2]);
/* Shared-inverse apply on the tensor cores (2-D Q2-Q1 batches with RAV_F32
 * rows and 8 right-hand sides; RAV_ERR_ARG otherwise).  On a uniform grid
 * with constant viscosity every interior subdomain of a level (vertex 2 .. N-2
 * on each axis) has the same local system, hence the same owned rows of
 * L_i^{-1} (Eq. 13).  With enable != 0 the call checks each (problem, level)
 * of the batch: where every interior subdomain's stored rows equal those of
 * the subdomain at vertex (2, 2) to within two units in the last place of
 * their largest entry, that level's interior subdomains are applied as one
 * small GEMM per 16 subdomains x 8 right-hand sides on the tensor cores
 * (tcgen05.mma kind::tf32, the fp32 operands split into tf32 high and low
 * parts, three products, fp32 accumulation: about 2^-20 relative error per
 * product), reading one copy of the rows instead of one per subdomain; the
 * boundary subdomains, and every subdomain of the other levels, stay on the
 * fp32 CUDA-core apply.  Synchronises the stream; drops the captured cycle.
 * Results differ from the CUDA-core apply by the rounding of the split
 * operands and the order of additions.  A tensor-core wait that gives up is
 * reported by solve_batched as RAV_ERR_TIMEOUT.  enable = 0 returns to the
 * CUDA-core apply.  batch_tensor_apply_levels returns how many (problem,
 * level) pairs use it (or RAV_ERR_ARG). */
int batch_set_tensor_apply(rav_batch* bt, int enable, rav_stream stream);
int batch_tensor_apply_levels(const rav_batch* bt);

/* FP32 residuals on the depths below the finest of a batch (enable = 1; 0
 * returns to fp64): there r = b - L x (Eq. 10) for every right-hand side uses
 * the operator values and x rounded to fp32 (x converted before each
 * residual), products summed in fp32 and r = b - sum formed in fp64; the
 * finest depth's residual, which measures convergence, and the coarse solves
 * stay fp64.  The single-problem counterpart is rav_set_coarse_residual_f32.
 * Allocates fp32 copies of those levels' operators and x, synchronises the
 * stream and drops the captured cycle.  RAV_ERR_ARG for other values.
 * batch_coarse_residual_f32 returns 1 when it is on, 0 when off.  The paper
 * has no counterpart. */
int batch_set_coarse_residual_f32(rav_batch* bt, int enable, rav_stream stream);
int batch_coarse_residual_f32(const rav_batch* bt);

/* FP32 grid transfers of a batch (FP32 rows, Q2-Q1; enable = 1; 0 returns to
 * fp64): the restriction reads the residual's fp32 copy (the one the apply
 * reads), the prolongation an fp32 copy of the coarse x (one conversion
 * kernel per transfer); fp32 weights and sums, b of the coarser level and
 * the update of x in fp64.  The single-problem counterpart is
 * rav_set_transfers_f32.  Allocates fp32 weight tables and coarse x copies,
 * synchronises the stream and drops the captured cycle.  RAV_ERR_ARG for
 * other values or another storage or element.  batch_transfers_f32 returns 1
 * when it is on, 0 when off.  The paper has no counterpart. */
int batch_set_transfers_f32(rav_batch* bt, int enable, rav_stream stream);
int batch_transfers_f32(const rav_batch* bt);

/* Timing hook of the batch, with the kernel classes of rav_profile_enable.
 * While enabled (on != 0) batch_vcycle and solve_batched launch phase by phase
 * instead of replaying the graph, and every phase launch is bracketed by CUDA
 * events on the launching stream.  Enabling (or disabling) waits for the
 * device and clears the totals.  batch_profile_read waits for the recorded
 * events and returns, for (depth below the finest grid, class), the number of
 * bracketed phase launches and their summed duration in ms. */
int batch_profile_enable(rav_batch* bt, int on);
int batch_profile_read(rav_batch* bt, int depth, int kind, int64_t* launches, double* total_ms);
/* One V(nu_pre, nu_post) cycle of every problem and right-hand side; x_dev[p]
 * updated in place, b_dev[p] read.  Synchronises the stream before rebinding
 * changed vector pointers. */
int batch_vcycle(rav_batch* bt, double* const* x_dev, const double* const* b_dev, int nu_pre, int nu_post,
                 rav_stream stream);
/* Stationary batched multigrid (opts->outer must be 0) until every problem
 * and right-hand side has ||r_k||/||r_0|| <= tol or maxit cycles are done;
 * iters_host[p * nrhs + k] = cycles that (p, k) needed (-1: not reached),
 * ratios_host[p * nrhs + k] = its last ratio.  Host-driven, one
 * synchronisation per cycle.  Returns RAV_ERR_NOT_CONVERGED if any (p, k)
 * missed the tolerance. */
int solve_batched(rav_batch* bt, double* const* x_dev, const double* const* b_dev, const rav_solve_opts* opts,
                  int* iters_host, double* ratios_host, rav_stream stream);

/* Timing hook.  Kernel classes: 0 subdomain apply (also each MV colour
 * sweep), 1 residual, 2 restriction, 3 prolongation, 4 coarse solve.  After
 * rav_profile_enable(mg, mask, level), every launch of a class whose bit is set
 * in mask, on the given level (-1: all levels), is bracketed by a pair of CUDA
 * events recorded on its launching stream.  Enabling clears the totals;
 * mask = 0 stops recording.  rav_profile_read waits for the recorded events
 * and returns, for (level, class), the number of bracketed launches and their
 * summed duration in ms since the last enable. */
int rav_profile_enable(rav_mg* mg, unsigned kind_mask, int level);
int rav_profile_read(rav_mg* mg, int level, int kind, int64_t* launches, double* total_ms);

/* Number of kernels the solve path of this library (residuals, subdomain
 * applies, transfers, coarse solves, Krylov vector updates) has launched in
 * this process so far; set-up kernels are not counted. */
int64_t rav_kernel_launches(void);

/* Measured FP64 fused multiply-add throughput of the current device in
 * TFLOP/s (2 flops per FMA), the denominator of the fp64-bound kernels'
 * rooflines: 10 timed launches (CUDA events on stream) of a kernel that runs 8
 * independent FMA chains of 4,096 steps in each of 256 threads x 8 blocks per
 * SM.  Synchronises the stream.  The paper has no counterpart. */
int rav_fp64_fma_rate(double* tflops_host, rav_stream stream);

/* Measured rate in GB/s of a plain read of `bytes` bytes (rounded down to 16)
 * on the current device: a coalesced grid-stride kernel of 16-byte
 * evict-first loads, 8 x 256 threads per SM, after an L2 flush (a write of
 * twice the L2 size), the mean of 10 timed launches (CUDA events on stream)
 * after a warm-up.  A memory-bound kernel that moves `bytes` can be set
 * against it: at tens to hundreds of MB the rate of such a short read stays
 * well below the large-copy bandwidth (launch, ramp-up and tail).  Allocates
 * and frees bytes + 2 x L2 of device memory; synchronises the stream.
 * RAV_ERR_ARG for bytes outside [16, 64 GiB].  The paper has no counterpart. */
int rav_hbm_read_rate(int64_t bytes, double* gbs_host, rav_stream stream);

const char* rav_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* RAVANKA_H */
