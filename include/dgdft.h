/* libdgdft: the data-parallel hot path of discontinuous Galerkin DFT
 * (DGDFT, Sec. II.A of "DGDFT on the Sunway TaihuLight", arXiv 2003.00407)
 * on one NVIDIA GB300 (sm_103a).
 *
 *   dgdft_alb_generate  per-element adaptive local basis: lowest eigenpairs
 *                       of the local Kohn-Sham Hamiltonian on each extended
 *                       element Q_k (Eq. LocalKS) by Chebyshev-filtered
 *                       subspace iteration (Alg. CheFSI), restricted to E_k
 *                       and truncated by SVD (Sec. II.A.1).
 *   dgdft_dg_assemble   interior-penalty DG Hamiltonian blocks (Eq.
 *                       DGHamiltonian) between each element and its stencil
 *                       neighbours.
 *   dgdft_alb_grad      Fermi-smeared band energy of the local problems and
 *                       its Hellmann-Feynman gradient with respect to V_eff
 *                       and the atom positions (local analogue of Eq. hfforce).
 *   dgdft_apply_hamiltonian / dgdft_chebyshev_filter
 *                       the hot operator alone (Eq. LocalKS; Alg. CheFSI step 2).
 *
 * Conventions
 *   - Grid functions are stored [z][y][x] (x fastest).  A block of n vectors
 *     on Q_k is [n][N_k] with N_k = Qx*Qy*Qz.  "Packed" buffers hold the
 *     blocks of elements 0..M-1 back to back: element k starts after the
 *     blocks of elements 0..k-1 (sizes from the element's own counts).
 *   - Problem description arrays (geometry, atoms, counts) are HOST memory,
 *     read during the call.  Data arrays (v_extra, results, blocks, grads)
 *     are DEVICE memory owned by the caller unless DGDFT_HOST_BUFFERS is set
 *     in params.flags, in which case they are host memory and the library
 *     stages them through its own device workspace (copies inside the call).
 *   - All calls are ordered on `stream` and synchronise it before returning
 *     (the iteration count depends on device-side convergence tests).
 *   - No call traps or aborts: every failure is a status code; the message of
 *     the last failure is returned by dgdft_last_error.  Device loops are
 *     bounded by max_iter.
 *   - A context owns the device workspace (grown on demand, freed by
 *     dgdft_ctx_destroy) and is not thread safe: use one context per thread.
 */
#ifndef DGDFT_H
#define DGDFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgdft_ctx dgdft_ctx;
typedef void* dgdft_stream; /* a cudaStream_t; NULL = the legacy default stream */

enum dgdft_status {
  DGDFT_OK = 0,
  DGDFT_INVALID_ARG = 1,    /* host-side argument check failed; nothing ran */
  DGDFT_OUT_OF_MEMORY = 2,  /* workspace allocation failed */
  DGDFT_NOT_CONVERGED = 3,  /* results written; some element hit max_iter (see status[]) */
  DGDFT_CHOLESKY_FAIL = 4,  /* Cholesky-QR failed even with a shift (see status[]) */
  DGDFT_BAD_INPUT = 5,      /* NaN/Inf found in v_extra or produced by the solve */
  DGDFT_TIMEOUT = 6,        /* reserved: a bounded device wait gave up */
  DGDFT_CUDA_ERROR = 7,     /* a CUDA call failed; message in dgdft_last_error */
  DGDFT_UNSUPPORTED = 8     /* valid but outside the library's limits (sizes, radices) */
};

enum dgdft_precision {
  DGDFT_FP64 = 0,  /* filter, orthonormalisation and Rayleigh-Ritz in FP64 */
  DGDFT_MIXED = 1  /* FP32 filter and subspace steps with FP64 small solves,
                      then one FP64 Rayleigh-Ritz sweep */
};

enum dgdft_solver {
  DGDFT_CHEFSI = 0,  /* Chebyshev-filtered subspace iteration (Alg. CheFSI), both precisions */
  DGDFT_LOBPCG = 1   /* LOBPCG with the Teter preconditioner (Alg. LOBPCG, Eqs. 3-5): DGDFT_FP64, the
                        same n_blk <= 32 in every element (the projected problem has 3 n_blk <= 96) */
};

enum dgdft_flags {
  DGDFT_HOST_BUFFERS = 1  /* data arrays are host memory (see Conventions) */
};

/* Statement of the problem (Sec. II.A: element partition, extended
 * elements, V_eff, Kleinman-Bylander projectors).  Host memory. */
typedef struct {
  int n_dom;                 /* periodic domains (1 for a partitioned system) */
  const int* dom_n;          /* [n_dom][3] grid points (x, y, z) */
  const double* dom_h;       /* [n_dom][3] spacing (bohr) */
  const int64_t* dom_voff;   /* [n_dom] first point of each domain in v_extra / grad_v */
  const double* v_extra;     /* DATA: V_eff minus the wells on all domains, or NULL (= 0) */
  int n_elem;                /* M */
  const int* elem_dom;       /* [M] */
  const int* elem_E0;        /* [M][3] first grid point of E_k */
  const int* elem_En;        /* [M][3] extent of E_k */
  const int* elem_Qn;        /* [M][3] extent of Q_k, centred on E_k (Qn-En even, Qn <= dom_n) */
  const int* neighbors;      /* [M][n_stencil] element ids; slot 0 = self, then faces
                                -x,+x,-y,+y(,-z,+z), then (9 slots) xy corners; -1 = none */
  int n_stencil;             /* 1, 3, 5, 7 or 9 */
  int n_atoms;
  const int* atom_dom;       /* [n_atoms] */
  const double* atom_pos;    /* [n_atoms][3] bohr */
  const double* well_depth;  /* [n_atoms] D_I: V_I(r) = -D_I exp(-d^2/2w^2) tau(d/r_cut) */
  const double* well_width;  /* [n_atoms] w_I */
  int n_proj_per_atom;       /* 0, 1 (s) or 4 (s, px, py, pz) */
  const double* proj_gamma;  /* [n_atoms][n_proj_per_atom] gamma_{I,l} (Ha) */
  const double* proj_width;  /* [n_atoms] sigma_I of b = N exp(-d^2/2 sigma^2) tau (p: times d_alpha) */
  double r_cut;              /* support radius; tau(s) = (1-s^2)^3 for s < 1, each domain side >= 2 r_cut */
} dgdft_problem;

/* Solver parameters (Alg. CheFSI).  Host memory. */
typedef struct {
  const int* n_eig;          /* [M] eigenpairs J_k */
  const int* n_alb;          /* [M] ALBs kept after the SVD (<= n_eig) */
  const int* n_blk;          /* [M] filter block (n_eig <= n_blk <= 96), or NULL for the
                                rule n_eig + max(4, ceil(n_eig/10)) rounded up to 8 */
  int cheb_degree;           /* filter order m >= 2 */
  double tol;                /* residual tolerance ||H x - lambda x|| (dV norm) of the first n_eig
                                Ritz pairs: DGDFT_FP64 iterates until every element meets it (else
                                status NOT_CONVERGED at max_iter); DGDFT_MIXED applies it to the FP32
                                stage, whose residuals stop at the FP32 rounding floor (see resid) */
  double tol_mixed;          /* DGDFT_MIXED: the FP32 stage stops at this residual or
                                when FP32 rounding stalls it; 0 = 1e-6 */
  int max_iter;              /* cap on filter passes per precision stage */
  int lanczos_steps;         /* steps of the upper-bound estimate (0 = 10) */
  int precision;             /* dgdft_precision */
  uint64_t seed;             /* SplitMix64 state of the random start */
  int flags;                 /* dgdft_flags */
  const double* x0;          /* DATA, optional warm start (NULL = random start): packed [n_eig][N] per
                                element, the layout of dgdft_alb_result.eigvec (e.g. the eigenvectors
                                of a previous call with a slightly different V_eff, as in the inner SCF
                                iterations of Sec. III).  Its n_eig vectors replace the first n_eig of
                                the start block (FP32-rounded in DGDFT_MIXED); the guard vectors keep
                                the SplitMix64 start.  Need not be orthonormal (CholQR2 follows). */
  int solver;                /* dgdft_solver (0 = CheFSI); cheb_degree and lanczos_steps apply to CheFSI */
} dgdft_alb_params;

/* Results of dgdft_alb_generate (DATA arrays; caller allocated).  Sizes in
 * scalars from dgdft_alb_query_sizes; L = max_k n_blk padded as returned. */
typedef struct {
  double* eigval;   /* [M][L] Ritz values, ascending (first n_blk valid) */
  double* resid;    /* [M][L] residual norms of the Ritz pairs.  DGDFT_MIXED: those of the final
                       FP64 Rayleigh-Ritz on the FP32-filtered subspace, at the FP32 rounding floor
                       (about 2e-5 on 32x32x48 grids); they are made of high-energy components, so
                       the eigenvalue error is of order resid^2 / ||H||, not resid */
  double* sing;     /* [M][L] singular values of the restricted block (first n_eig) */
  double* coef;     /* [M][L][L] C_k: ALB = Phi_E C_k (first n_eig rows, n_alb cols) */
  double* alb;      /* packed [n_alb][NE] per element: ALB values on E_k, dV-orthonormal */
  double* eigvec;   /* packed [n_eig][N] per element: eigenvectors on Q_k, dV-orthonormal */
  int* iters;       /* [M] filter passes (both stages in mixed mode) */
  int* status;      /* [M] per-element status: 0 ok, or a dgdft_status */
  double* history;  /* HOST, optional (NULL): [max_iter + 2] largest residual over the still-active
                       elements after the start-up Rayleigh-Ritz (entry 0) and after each filter
                       pass of the first stage; unused entries are set to -1 */
} dgdft_alb_result;

/* Sizes (in scalars) of the result arrays for a problem:
 * out[0] = L (row length of eigval/resid/sing and the side of coef),
 * out[1] = size of alb, out[2] = size of eigvec, out[3] = M*L*L (coef),
 * out[4] = total points of all domains (grad_v), out[5] = n_stencil*M*L*L (blocks). */
int dgdft_alb_query_sizes(const dgdft_problem* prob, const dgdft_alb_params* params, int64_t out[6]);

/* Creates a context on CUDA device `device` (uploads the transform twiddle tables, sets the kernels'
 * shared-memory limits).  *ctx receives the handle, or NULL on failure: DGDFT_CUDA_ERROR when the device
 * is missing or unusable (message from dgdft_last_error(NULL)).  dgdft_ctx_destroy frees every device
 * and pinned buffer the context grew; NULL is ignored. */
int dgdft_ctx_create(dgdft_ctx** ctx, int device);
void dgdft_ctx_destroy(dgdft_ctx* ctx);
/* Message of the last failure on ctx; with ctx == NULL, of the last failure on
 * this thread that had no context (e.g. dgdft_ctx_create). */
const char* dgdft_last_error(const dgdft_ctx* ctx);

/* Number of CUDA kernel launches this library has issued since it was loaded
 * (all contexts, all threads).  For accounting in benchmarks. */
int64_t dgdft_kernel_launches(void);

/* The stopping test that dgdft_alb_generate applies to one element after each CheFSI pass (Alg. CheFSI:
 * iterate until the residuals of the wanted Ritz pairs meet the tolerance), exported so that callers and
 * tests can check the rule on a residual history without a GPU.  Host only, no device work.
 *   max_resid  largest residual ||H x - theta x|| (dV norm) of the first n_eig Ritz pairs after this pass
 *   tol        DGDFT_FP64 stage: leave at max_resid <= tol (a non-finite residual also ends the stage)
 *   tol_mixed  FP32 stage (mixed != 0): leave at max_resid <= tol_mixed, or after two consecutive passes
 *              that each cut the residual by less than 20% and end at most at 32 * 2^-24 * |b_up|
 *              (the FP32 rounding floor of H with spectrum bound b_up); stagnation above that level
 *              does not end the stage (the element runs on to max_iter and reports NOT_CONVERGED)
 *   prev_resid, stall  per-element state, updated in place; start with *prev_resid = 1e300, *stall = 0
 * Returns 1 when the element leaves the stage, 0 when it continues, -DGDFT_INVALID_ARG for null state. */
int dgdft_stage_converged(double max_resid, double tol, double tol_mixed, int mixed, double b_up, double* prev_resid,
                          int* stall);

/* Gram matrices of FP32 vector blocks on the tensor cores: for every block k,
 *   G_k[i][j] = dV_k sum_p X_k[i][p] Y_k[j][p]      (i < nx[k], j < ny[k], p < np[k])
 * the overlap X^T X of the Cholesky-QR step and the projection X^T (H X) of the Rayleigh-Ritz step of
 * Alg. CheFSI, as the FP32 stage of dgdft_alb_generate forms them (the same kernel).  Each input is split
 * into two TF32 parts (x = x_hi + x_lo); the products x_hi y_hi + x_hi y_lo + x_lo y_hi run on
 * tcgen05 tensor cores with FP32 accumulation over 512 points, the partial sums are added exactly
 * (two-sum) over 4096 points and in FP64 beyond.  Error: a few 2^-22 of dV_k sum_p |X_k[i][p]| |Y_k[j][p]|.
 *   n_blocks             number of blocks (0: nothing to do)
 *   nx, ny, np, dV       host arrays [n_blocks]: rows of X_k (0..96), rows of Y_k (0..96), points, volume element
 *   X, Y                 device FP32: X_k row-major [nx[k]][np[k]] starting at X + x_off[k] (Y likewise; Y may be X)
 *   x_off, y_off         host arrays [n_blocks] of element offsets (>= 0)
 *   G                    device FP64 [n_blocks][ldg][ldg], overwritten (entries outside the nx x ny block are 0)
 *   ldg                  >= every nx[k] and ny[k]
 *   stream               CUDA stream; the call returns after the work on it has completed
 * Uses the context's grow-only workspace for the block table.  Errors: DGDFT_INVALID_ARG (null pointers,
 * counts or offsets out of range), DGDFT_CUDA_ERROR (including a bounded tensor-core wait that ran out). */
int dgdft_gram_fp32(dgdft_ctx* ctx, int n_blocks, const int* nx, const int* ny, const int* np, const double* dV,
                    const float* X, const int64_t* x_off, const float* Y, const int64_t* y_off, double* G, int ldg,
                    dgdft_stream stream);

/* Subspace rotation of FP32 vector blocks on the tensor cores: for every block k,
 *   Z_k[j][p] = sum_i W_k[i][j] X_k[i][p]          (j < nout[k], i < nin[k], p < np[k])
 * the X <- X U^-1 step of Cholesky-QR and the X <- X C step of Rayleigh-Ritz of Alg. CheFSI, on the
 * tensor cores (dgdft_alb_generate's FP32 stage applies the same rotations with a CUDA-core kernel, which
 * measured faster on the sheet elements).  X and W are split into two TF32 parts each
 * (3xTF32 products on tcgen05 tensor cores, FP32 accumulation over the nin terms).  Error: a few 2^-22
 * of sum_i |W_k[i][j]| |X_k[i][p]|.
 *   n_blocks               number of blocks (0: nothing to do)
 *   nin, nout, np          host arrays [n_blocks]: input vectors (0..96), output vectors (0..96), points
 *   X                      device FP32: X_k row-major [nin[k]][np[k]] at X + x_off[k]
 *   W                      device FP64 [n_blocks][ldw][ldw], row i of block k = input vector i
 *   Z                      device FP32: Z_k [nout[k]][np[k]] at Z + z_off[k]; Z may be X (in place, same offsets)
 *   x_off, z_off           host arrays [n_blocks] of element offsets (>= 0)
 *   stream                 CUDA stream; the call returns after the work on it has completed
 * Uses the context's grow-only workspace for the block table.  Errors: DGDFT_INVALID_ARG (null pointers,
 * counts or offsets out of range), DGDFT_CUDA_ERROR (including a bounded tensor-core wait that ran out). */
int dgdft_rotate_fp32(dgdft_ctx* ctx, int n_blocks, const int* nin, const int* nout, const int* np, const float* X,
                      const int64_t* x_off, const double* W, int ldw, float* Z, const int64_t* z_off,
                      dgdft_stream stream);

/* ALB generation for all elements in one batched solve: the lowest n_eig eigenpairs of each local
 * Hamiltonian (Eq. LocalKS) by Chebyshev-filtered subspace iteration (Alg. CheFSI: Lanczos upper bound,
 * scaled Chebyshev filter, Cholesky-QR, Rayleigh-Ritz; in DGDFT_MIXED an FP32 stage, then one FP64
 * Rayleigh-Ritz sweep), their restriction to E_k and the SVD truncation to n_alb ALBs (Sec. II.A.1).
 * result arrays are caller-allocated with the sizes of dgdft_alb_query_sizes; eigvec may be NULL (the
 * eigenvectors then stay in the context for dgdft_dg_assemble / dgdft_alb_grad).  Returns DGDFT_OK, or
 * DGDFT_NOT_CONVERGED / DGDFT_CHOLESKY_FAIL / DGDFT_BAD_INPUT with every element's own status in
 * result->status and all outputs filled; DGDFT_INVALID_ARG / DGDFT_UNSUPPORTED before any GPU work;
 * DGDFT_OUT_OF_MEMORY / DGDFT_CUDA_ERROR. */
int dgdft_alb_generate(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* params,
                       dgdft_alb_result* result, dgdft_stream stream);

/* DG blocks from a result of dgdft_alb_generate (eigvec, coef, alb used).
 * blocks: DATA [M][n_stencil][L][L]; block (k, s) has rows = test ALBs of
 * element k and columns = trial ALBs of neighbors[k][s] (Eq. DGHamiltonian).
 * alpha is the penalty (Ha bohr).  The nonlocal coupling of a pair goes to the
 * first slot naming it; faces along axes where E spans its domain are skipped. */
int dgdft_dg_assemble(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* params,
                      const dgdft_alb_result* result, double alpha, double* blocks, dgdft_stream stream);

/* The two halves of dgdft_dg_assemble, for callers that distribute the elements (Sec. II.B: the
 * elements are split among processes, and building H^DG needs the face and projector data of the
 * neighbouring elements, which are exchanged point to point).  An element's DG ingredients depend only
 * on its own ALBs; the blocks of element k need the ingredients of k and of its stencil neighbours.
 *
 * Layout of the ingredients of a problem (DATA arrays, scalars):
 *   kv      [M][L][L]   kinetic + V_eff part of the diagonal block (L as in dgdft_alb_query_sizes)
 *   traces  element k's record at tr_off[k]: [6 faces][2][n_alb_k][F_k] -- face = 2*axis + (1 on the
 *           high side), kind 0 = value, 1 = outward-axis derivative of the ALB interpolant on the face
 *           plane half a spacing outside E_k; F_k = the element's largest face (points), a face's points
 *           run over the two transverse axes of E_k (lower axis fastest); faces along axes the stencil
 *           does not name, or along which E_k spans its domain, are zero; records of elements without
 *           such faces are empty
 *   proj    element k's record at pe_off[k]: [n_alb_k][P_k], P_k projector columns of the atoms whose
 *           support meets E_k, in ascending atom order, n_proj_per_atom columns each
 * dgdft_dg_query_layout (host only) fills tr_off[M+1] and pe_off[M+1] (cumulative, last entry = total).
 * Records depend only on the element's own geometry and the atoms, so the record of an element is the
 * same in every problem that contains it: a record computed by one process can be copied into the
 * arrays of another process's problem at that problem's offsets.
 *
 * dgdft_dg_ingredients fills kv/traces/proj from a dgdft_alb_generate result (like dgdft_dg_assemble).
 * dgdft_dg_blocks forms blocks [M][n_stencil][L][L] from ingredients; the blocks of an element are
 * valid when its own record and those of its neighbours are filled (a neighbour id -1 gives zero
 * blocks).  Status codes as dgdft_dg_assemble; dgdft_dg_assemble equals the two calls in a row. */
int dgdft_dg_query_layout(const dgdft_problem* prob, const dgdft_alb_params* params, int64_t* tr_off,
                          int64_t* pe_off);
int dgdft_dg_ingredients(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* params,
                         const dgdft_alb_result* result, double* kv, double* traces, double* proj,
                         dgdft_stream stream);
int dgdft_dg_blocks(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* params, const double* kv,
                    const double* traces, const double* proj, double alpha, double* blocks, dgdft_stream stream);

/* Parameters of dgdft_dg_eigensolve.  Host memory. */
typedef struct {
  int n_states;              /* lowest eigenpairs wanted */
  int n_blk;                 /* filter block, n_states <= n_blk <= min(96, N_b) */
  int cheb_degree;           /* filter order m >= 2 */
  double tol;                /* residual ||H c - eps c|| (Euclidean) of the first n_states Ritz pairs */
  int max_iter;              /* cap on filter passes */
  int lanczos_steps;         /* steps of the upper-bound estimate (0 = 10) */
  uint64_t seed;             /* SplitMix64 state of the random start (element index 0) */
} dgdft_dg_solve_params;

/* Lowest eigenpairs of the assembled DG Hamiltonian (Eq. DGEigenvalue; the ALB basis is orthonormal, so
 * the problem is the standard symmetric one) by Chebyshev-filtered subspace iteration (Alg. CheFSI, the
 * paper's solver for H^DG), FP64.  H^DG is applied from `blocks` (DATA [M][n_stencil][L][L] as written
 * by dgdft_dg_assemble: block (k, s) couples the test ALBs of element k with the trial ALBs of
 * neighbors[k][s]), never formed.  The basis index runs over the elements in order, n_alb[k] functions
 * each (N_b = sum n_alb).  Outputs (DATA): eigval [n_blk] ascending, resid [n_blk], eigvec [n_blk][N_b]
 * (rows orthonormal; may be NULL), iters [1] filter passes.  Returns DGDFT_OK, DGDFT_NOT_CONVERGED
 * (outputs written), DGDFT_CHOLESKY_FAIL, DGDFT_BAD_INPUT, DGDFT_INVALID_ARG (sizes), DGDFT_UNSUPPORTED
 * (N_b >= 2^24), DGDFT_OUT_OF_MEMORY, DGDFT_CUDA_ERROR. */
int dgdft_dg_eigensolve(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* params,
                        const double* blocks, const dgdft_dg_solve_params* solve, double* eigval, double* resid,
                        double* eigvec, int* iters, dgdft_stream stream);

/* Electron density, band energy and Hellmann-Feynman forces of the DG solution (Eq. density with the
 * diagonal blocks of the density matrix, Eq. densitymatrix; Eq. DGvar on the DG eigenpairs, which is the
 * band energy sum_i 2 f_i eps_i; Eq. hfforce for the wells and projectors of this model, at fixed ALBs).
 *   result     the dgdft_alb_generate result whose ALBs (result->alb) span the DG basis
 *   eigval     DATA [n] DG eigenvalues (e.g. from dgdft_dg_eigensolve), eigvec DATA [n][N_b] their
 *              orthonormal coefficient rows in the ALB basis (elements in order, n_alb[k] each)
 *   n          states used (1..96); f_i Fermi-Dirac at kT with mu fixed by sum_i 2 f_i = n_electrons
 *   rho        DATA [total points of all domains]: sum_i 2 f_i psi_i(r)^2 at the points of every E_k (0
 *              elsewhere)
 *   energy_mu  DATA [2]: the band energy and mu
 *   grad_R     DATA [n_atoms][3] or NULL: dE/dR_I at fixed ALBs (the force is its negative), including the
 *              term that keeps the electron count fixed
 * Device buffers only (DGDFT_HOST_BUFFERS returns DGDFT_UNSUPPORTED).  DGDFT_BAD_INPUT when the highest of
 * the n states is occupied (f >= 1e-12). */
int dgdft_dg_density(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* params,
                     const dgdft_alb_result* result, const double* eigval, const double* eigvec, int n,
                     double n_electrons, double kT, double* rho, double* energy_mu, double* grad_R,
                     dgdft_stream stream);

/* Band energy E_k = sum_j 2 f_j lambda_j (f Fermi-Dirac at kT, mu_k fixed by
 * n_electrons[k], a host array) and its gradient: energy DATA [M],
 * grad_v DATA [total points of all domains] (dE/dV at each grid point,
 * including dV), grad_R DATA [n_atoms][3].  Uses eigval and eigvec. */
int dgdft_alb_grad(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* params,
                   const dgdft_alb_result* result, double kT, const double* n_electrons, double* energy,
                   double* grad_v, double* grad_R, dgdft_stream stream);

/* The hot operator: Y = H X for packed FP64 (precision DGDFT_FP64) or FP32
 * (DGDFT_MIXED) blocks of params.n_blk vectors per element (device memory).
 * A non-finite v_extra on some Q_k returns DGDFT_BAD_INPUT naming element k. */
int dgdft_apply_hamiltonian(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* params,
                            const void* X, void* Y, dgdft_stream stream);

/* One Chebyshev filter pass Y = p_m(H) X of degree params.cheb_degree
 * (Alg. CheFSI step 2: [b_low, b_up] mapped to [-1, 1], scaled at a0) with
 * per-element bounds[k] = {a0, b_low, b_up} (host [M][3]), on packed blocks as
 * in dgdft_apply_hamiltonian.  X is not modified. */
int dgdft_chebyshev_filter(dgdft_ctx* ctx, const dgdft_problem* prob, const dgdft_alb_params* params,
                           const double* bounds, const void* X, void* Y, dgdft_stream stream);

/* Allocation-free variant of dgdft_apply_hamiltonian for FP32 blocks
 * (params.precision must be DGDFT_MIXED): Y = H X with no device allocation at
 * all, for callers that cannot call cudaMalloc/cudaFree -- hosts whose device
 * memory is reserved entirely by another allocator, or latency-critical code
 * that cannot accept the device-wide synchronisation of cudaMalloc/cudaFree.
 * The paper has no counterpart; it is a deployment aid.
 *   - No context: every scratch table (element tables, V_eff on Q, projector
 *     factor tables) is placed in one fixed 24 MiB device array inside the
 *     library, which every GPU that loads the library holds until exit.  A
 *     problem that needs more returns DGDFT_UNSUPPORTED (message: the bytes it
 *     needs) before anything runs; so does a Q shape the fused FP32 kernel does
 *     not cover.
 *   - The first call on a device (the current one) looks up the array's device
 *     address and uploads the FFT twiddles; make that first call before any
 *     stream capture.
 *   - All calls share the array and it keeps the last call's contents: calls
 *     that overlap on the GPU (other streams or host threads) race on it.
 *   - X, Y and problem->v_extra are caller-owned device buffers laid out as in
 *     dgdft_apply_hamiltonian; the call synchronises `stream` before returning.
 *   - A non-finite v_extra on some Q_k returns DGDFT_BAD_INPUT naming element k
 *     (Y of that element is then not valid).
 *   - Errors are reported by dgdft_last_error(NULL). */
int dgdft_apply_hamiltonian_noalloc(const dgdft_problem* prob, const dgdft_alb_params* params, const float* X,
                                    float* Y, dgdft_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* DGDFT_H */
