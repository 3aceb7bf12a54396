/*
 * dg_poisson.h -- C ABI of the GB300 library for the exchange-build hot path of
 * the discontinuous-Galerkin Hartree-Fock method of arXiv 2510.21213
 * ("Fast adaptive discontinuous basis sets for electronic structure").
 *
 * What the library computes (citations are to the paper):
 *
 *   For every source f given at the Gauss-Legendre nodes of a uniform box mesh
 *   of degree-p nodal elements (Sec. 6.2, eq. density_approx; the nodes double
 *   as the quadrature rule), the solution v of the SIPDG-discretised Poisson problem
 *       -Lap v = 4 pi f  in Omega,
 *        v(r)  = int_Omega f(r') / |r - r'| dr'   on the boundary of Omega
 *   (Sec. 6.3; the boundary integral is the grid's Gauss quadrature), with the
 *   SIPDG bilinear form of Sec. 3.4 (eq. sip_bilinear) and the penalty of
 *   Sec. 3.5 (eqs. Cprop, Csquared, pen_poly), solved by conjugate gradients
 *   preconditioned with hp-multigrid: polynomial coarsening to degree 1, then
 *   geometric coarsening on the nested hierarchy (Sec. 6.4).
 *
 *   Level hierarchy: degree p -> floor(p/2) down to 1 on the fine mesh, then
 *   n -> n/2 (all axes) while every n is even and the level has more than 512
 *   unknowns; the last level is solved exactly (dense inverse).
 *
 *   dg_exchange_build applies this to the Hartree density rho = sum_k psi_k^2
 *   (Sec. 2.3.1 eq. HF; Sec. 6.1.1 eq. hartree_poisson) and to every occupied
 *   pair density psi_i psi_j (Sec. 6.1.2 eq. fock_poisson), then contracts
 *   K_ij = sum_q W_q psi_i(q) sum_s psi_s(q) v_sj(q) on the quadrature grid
 *   (eq. fock_exchange with phi_i -> psi_i, u -> psi_j), and returns
 *   E_H = 1/2 sum_q W_q rho v_H and E_X = -1/2 tr K (HF energy, Sec. 2.3.1).
 *
 * Readings of points the paper leaves open (same in every entry point):
 *   - Dirichlet data are imposed weakly by symmetric Nitsche terms
 *     -u d_n v - d_n u v + sigma u v on boundary faces (paper: "inhomogeneous
 *     Dirichlet", weak form unstated).
 *   - sigma = (p+1)^2 / (eps h) (penalty_form 0) or the literal
 *     (p+1)^2 / (eps h^2) (penalty_form 1); eps = 1/8 by default (Sec. 3.5).
 *   - Each distinct pair (i <= j) is solved once, v_ij = v_ji.
 *
 * Layouts. All node-valued arrays are element-blocked: element index
 * e = ex + nx*(ey + ny*ez), and inside an element the (p+1)^3 nodes are
 * lexicographic, x fastest: local = a + (p+1)*(b + (p+1)*c). A field occupies
 * Nq = nx*ny*nz*(p+1)^3 contiguous doubles; a batch of fields is [B][Nq].
 * Orbital pairs are ordered upper-triangular row-major: (0,0),(0,1),...,(0,N-1),
 * (1,1),...
 *
 * Ownership. The caller owns every input and output buffer. "dev" pointers are
 * CUDA device memory of the current device, "host" pointers are host memory.
 * The handle owns all workspace; it is allocated in dg_poisson_setup and grown
 * (never shrunk) the first time a larger batch is solved.
 *
 * Errors. Every int-returning call returns DG_OK (0) or a negative DG_ERR_*
 * code; no exception crosses the ABI. dg_error_string maps a code to text.
 * dg_last_error_detail(h) returns a message for the last failure on a handle.
 *
 * Concurrency. One handle per stream; calls on a handle are stream-ordered and
 * synchronise that stream before returning (results that land in host memory
 * are complete on return).
 */
#ifndef DG_POISSON_H
#define DG_POISSON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_OK 0
#define DG_ERR_INVALID_ARG (-1)
#define DG_ERR_CUDA (-2)
#define DG_ERR_NOT_CONVERGED (-3)
#define DG_ERR_BREAKDOWN (-4)
#define DG_ERR_NONFINITE (-5)
#define DG_ERR_TIMEOUT (-6)
#define DG_ERR_NO_MEMORY (-7)
#define DG_ERR_UNSUPPORTED (-8)

/* precision modes */
#define DG_PREC_FP64 0  /* every step in FP64 */
#define DG_PREC_MIXED 1 /* FP32 inner multigrid-PCG, FP64 dots, residuals and refinement */
#define DG_PREC_MIXED_LEARNED 2 /* as MIXED, initial guess and coarse correction from a network */

/* boundary-data routes */
#define DG_BC_DIRECT 0   /* direct Gauss-quadrature Coulomb sum (the definition, Sec. 6.3) */
#define DG_BC_GAUSSSUM 1 /* separable sum-of-Gaussians 1/r (Sec. 5.2) evaluated on the faces */

/* multigrid smoothers (the paper names none; Sec. 6.4 gives only the hierarchy) */
#define DG_SMOOTH_JACOBI 0  /* point Jacobi */
#define DG_SMOOTH_SCHWARZ 1 /* additive Schwarz on element patches with one node of overlap, exact
                               patch solves by fast diagonalisation */

/* Uniform hexahedral box mesh: box [lo, hi], n[d] elements along axis d,
 * tensor Gauss-Legendre nodal elements of degree p (1 <= p <= 8). */
typedef struct {
  double lo[3];
  double hi[3];
  int32_t n[3];
  int32_t p;
} dg_mesh_desc;

typedef struct {
  int32_t precision;     /* DG_PREC_* */
  double rtol;           /* target FP64 true relative residual ||b - A v||_2 / ||b||_2 */
  int32_t max_iter;      /* PCG iteration cap (per source, summed over refinements) */
  double penalty_eps;    /* eps of Sec. 3.5 (default 1/8) */
  int32_t penalty_form;  /* 0: (p+1)^2/(eps h); 1: (p+1)^2/(eps h^2) */
  int32_t bc_route;      /* DG_BC_* */
  double bc_tol;         /* relative accuracy of the Gaussian-sum 1/r (0 = precision default) */
  int32_t batch;         /* sources solved together (0 = library default) */
  int32_t smoother;      /* DG_SMOOTH_*: preconditioner inside the Chebyshev smoother */
  int32_t smoother_degree; /* Chebyshev degree of the multigrid smoother (default 4) */
  double cheb_range;     /* smoothing range lambda_max / lambda_min of the Chebyshev interval (default 10) */
  double inner_rtol;     /* MIXED: relative reduction of each FP32 inner solve (default 1e-4) */
  const char* nn_weights_path; /* MIXED_LEARNED: network weights file (NULL: set by dg_nn_set_params) */
  int32_t verbose;       /* 0 silent, 1 per-solve summary, 2 also per refinement round (stderr) */
  int32_t coarse_penalty; /* 0: each multigrid level uses the penalty of its own p and h;
                             1: every level uses the fine level's penalty (Galerkin-consistent hierarchy) */
  int32_t coarse_smoother_degree; /* Chebyshev degree on the levels below the finest (0 = smoother_degree) */
  int32_t p1_smoother;   /* smoother of the degree-1 levels below the finest: -1 = as `smoother`, else DG_SMOOTH_* */
  int32_t gauss_construction; /* Gaussian-sum 1/r: 0 = tabulated short sums (nonnegative least-squares fits,
                                 about 3-5x fewer terms), the trapezoidal rule where no table applies;
                                 1 = trapezoidal rule only */
  int32_t tc_smoother;   /* MIXED modes: Schwarz patch problems of the FP32 inner solve on the tensor cores
                            (TF32 tcgen05 MMA). 1 (default): on levels of degree 7 and 8, where it is
                            measured faster than the FP32 SIMT kernel; 2: also at degree 6; 0: off */
  int32_t nn_use_net;    /* MIXED_LEARNED: 1 (default) starts from the network's guess; 0 from the same
                            guess without the network (the prolongated degree-1 coarse solution, smoothed and
                            scaled), to measure what the network itself adds */
  int32_t device_loop;   /* PCG iterations driven from the device: 1: each launch of a captured graph runs
                            iterations in a conditional while-node that tests convergence on the device and
                            stops when a source converges, after which the host drops it and launches the
                            continuation (one host round trip per convergence event, results bit-identical
                            to 0); 0: two graph launches and one host read of the residual norms per
                            iteration; 2 (default): 1 for batches of at most 2^24 unknowns, else 0 */
} dg_solver_opts;

typedef struct {
  int32_t iters;             /* PCG iterations (inner iterations in MIXED modes) */
  int32_t outer_refinements; /* FP64 refinement steps (0 in FP64 mode) */
  int32_t status;            /* DG_OK, DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN or DG_ERR_NONFINITE */
  int32_t used_fallback;     /* 1 if a learned guess was rejected and the plain solver used */
  double rel_residual;       /* final FP64 true relative residual */
  double guess_rel_residual; /* FP64 relative residual of the initial guess (1 for the zero guess) */
  double self_energy;        /* Coulomb self-energy of the source, (f|f) = sum_q W_q f(q) v(q) (Sec. 2.3.1):
                                for a pair density f = psi_i psi_j the integral (ij|ij), for the density
                                rho = 2 E_H; FP64, from the returned v */
} dg_solve_stats;

typedef struct {
  int64_t Nq;          /* nodes (= unknowns) of the fine level */
  int32_t levels;      /* multigrid levels, fine to coarsest */
  int32_t level_n[16]; /* elements per axis (x) of each level */
  int32_t level_p[16]; /* degree of each level */
  int32_t coarse_dofs; /* unknowns of the coarsest (directly solved) level */
  int32_t n_gauss;     /* terms of the Gaussian-sum 1/r used for boundary data */
  double gauss_rmin, gauss_rmax; /* distance range on which that sum is accurate */
  double gauss_relerr; /* measured max relative error of the sum on that range */
  double sigma[3];     /* fine-level penalty per axis */
  int64_t workspace_bytes; /* device workspace currently held by the handle */
  int32_t n_gauss_fp32; /* terms of the FP32 Gaussian sum of the mixed modes (0 in FP64 mode) */
  double gauss_relerr_fp32; /* its measured max relative error */
  int32_t batch;        /* sources the solve calls process together (opts.batch, or the default that
                           fills about 8 GB of FP64 fine-level vectors) */
} dg_info;

typedef struct dg_ctx* dg_handle;

/* Fills *opts with defaults: FP64, rtol 1e-8, max_iter 500, eps 1/8,
 * penalty_form 0, Gaussian-sum boundary data, Schwarz smoother, Chebyshev
 * degree 4 over a smoothing range of 10, inner_rtol 1e-4, coarse_penalty 0. */
void dg_default_opts(dg_solver_opts* opts);

/* Builds the level hierarchy, 1-D operator tables, Chebyshev bounds, the
 * coarsest-level inverse and the boundary-data tables (step S0); copies them
 * to the device. mesh, opts: host structs, read only. *out receives a handle
 * to be released with dg_destroy. Errors: DG_ERR_INVALID_ARG for p outside
 * 1..8, non-positive sizes or an empty box; DG_ERR_UNSUPPORTED if the coarsest
 * level would exceed 4096 unknowns; DG_ERR_CUDA / DG_ERR_NO_MEMORY. */
int dg_poisson_setup(const dg_mesh_desc* mesh, const dg_solver_opts* opts, dg_handle* out);

/* Properties of a handle. info: host. */
int dg_get_info(dg_handle h, dg_info* info);

/* Node coordinates [Nq][3] and quadrature weights W_q [Nq] of the fine level
 * in the element-blocked order (host buffers, caller-allocated). Either
 * pointer may be NULL. */
int dg_node_coords(dg_handle h, double* xyz_host, double* w_host);

/* As dg_node_coords, from a mesh description alone (host computation, no
 * handle, no GPU). */
int dg_mesh_node_coords(const dg_mesh_desc* mesh, double* xyz_host, double* w_host);

/* Solves -Lap v_b = 4 pi f_b with Coulomb-quadrature Dirichlet data for B
 * sources (steps S1-S4 and S10 for a batch). f_dev: [B][Nq] source values at
 * the nodes (device, read only). v_dev: [B][Nq] solutions (device, written).
 * stats_host: [B] per-source statistics (host, may be NULL). cuda_stream: a
 * cudaStream_t (NULL = default stream). Returns DG_OK when every source
 * reached rtol; otherwise the worst per-source status (a non-converged source
 * still returns its best iterate). DG_ERR_NONFINITE if a source is not finite
 * (its v is set to zero). */
int dg_pair_solve_batch(dg_handle h, const double* f_dev, int64_t B, double* v_dev,
                        dg_solve_stats* stats_host, void* cuda_stream);

/* Exchange build for N orbitals psi_dev [N][Nq] (device, read only): the
 * Hartree solve, the N(N+1)/2 pair solves, the accumulation
 * W_j = sum_s psi_s v_sj, K = Psi^T diag(W_q) W and the energies.
 * K_host: [N*N] row-major K_ij (host). E_H, E_X: host scalars (may be NULL).
 * stats_host: [N(N+1)/2 + 1] (host, may be NULL): entry 0 is the Hartree
 * solve, then the pairs in the documented order; their self_energy fields
 * hold (rho|rho) = 2 E_H and the pair self-energies (ij|ij) of step S13
 * (Sec. 2.3.1, Sec. 6.1.2), from the pair potentials before they are
 * consumed by the accumulation. */
int dg_exchange_build(dg_handle h, const double* psi_dev, int32_t N, double* K_host, double* E_H,
                      double* E_X, dg_solve_stats* stats_host, void* cuda_stream);

/* Part of an exchange build, for sharding one system's sources over GPUs
 * (one handle per GPU, no communication inside the call). The sources are
 * numbered as in dg_exchange_build's stats: 0 = Hartree density, 1.. = the
 * pairs (i <= j) row-major; this call solves [src_begin, src_end) and returns
 * in K_partial_host [N*N] (host) their contribution sum_s psi_i (psi_s v_sj)
 * to K_ij (eq. fock_exchange, Sec. 6.1.2). The partial K of disjoint ranges
 * covering 0 .. N(N+1)/2 add up to dg_exchange_build's K (up to the summation
 * order); E_X = -1/2 tr of the sum. E_H (host, may be NULL) is set when the
 * range holds source 0 and is 0 otherwise. stats_host: [src_end - src_begin]
 * (may be NULL). An empty range returns K_partial = 0. DG_ERR_INVALID_ARG for
 * a range outside 0 .. N(N+1)/2 + 1. */
int dg_exchange_build_range(dg_handle h, const double* psi_dev, int32_t N, int64_t src_begin, int64_t src_end,
                            double* K_partial_host, double* E_H, dg_solve_stats* stats_host, void* cuda_stream);

/* Adaptively compressed exchange operator of the handle's last whole
 * dg_exchange_build (the compressed exchange the HF SCF of Sec. 7.2 applies;
 * V_X of Sec. 2.3.1 eq. exchange on the occupied space): for m trial vectors
 * U_dev [m][Nq] (device, FP64)
 *     Y_dev = V_X^ACE U = -W K_s^-1 (W^T diag(W_q) U),  K_s = (K + K^T) / 2,
 * with W_j = sum_s psi_s v_sj the build's exchange accumulation and K its
 * exchange matrix; Y_dev [m][Nq] (device). V_X^ACE has rank N, is symmetric
 * and negative semidefinite in the quadrature inner product and maps psi_i
 * to -W_i = V_X psi_i. DG_ERR_INVALID_ARG if the handle has no whole build
 * (a failed build or a dg_exchange_build_range call clears it) or N * m >
 * 4096; DG_ERR_BREAKDOWN if K_s is not positive definite. */
int dg_ace_apply(dg_handle h, const double* U_dev, int64_t m, double* Y_dev, void* cuda_stream);

/* Hartree and exchange actions on m trial functions (the operators of
 * Sec. 2.3.1 that an eigensolver applies; the same auxiliary-grid solves as
 * dg_exchange_build, Sec. 6.1, with a trial function in place of the second
 * orbital). For psi_dev [N][Nq] (device, read only, FP64) and trial values at
 * the fine-level nodes U_dev [m][Nq] (device, read only, FP64):
 *     JU[k](q) = v_H(q) u_k(q),               -lap v_H  = 4 pi sum_j psi_j^2
 *     XU[k](q) = -sum_j psi_j(q) v_jk(q),     -lap v_jk = 4 pi psi_j u_k
 * each v with its own Coulomb boundary data and solved to the handle's rtol.
 * JU_dev, XU_dev: [m][Nq] (device, written); either may be NULL to skip that
 * operator (the Hartree solve is made only for JU). The sum over j runs in
 * ascending j. Solves: (JU ? 1 : 0) + (XU ? N m : 0), numbered in that order
 * (the Hartree density first, then u_0 with psi_0 .. psi_{N-1}, then u_1 ...);
 * stats_host: one entry per solve (host, may be NULL). Applied to the
 * orbitals themselves, XU = -W of the exchange build and
 * <psi_i, XU_j> = -K_ij. Returns DG_OK when every solve reached rtol, else the
 * worst per-solve status (as dg_pair_solve_batch); DG_ERR_INVALID_ARG for N or
 * m < 1, m > 65535, more than 2^30 solves, a NULL psi_dev or U_dev, or both
 * outputs NULL. */
int dg_jk_apply(dg_handle h, const double* psi_dev, int32_t N, const double* U_dev, int64_t m, double* JU_dev,
                double* XU_dev, dg_solve_stats* stats_host, void* cuda_stream);

/* Exchange builds of nsys independent systems with their own meshes and
 * orbital counts (uneven sizes), as one call. meshes [nsys] (host), psi_devs
 * [nsys] device pointers to [Ns[i]][Nq_i], K_hosts [nsys] host pointers to
 * [Ns[i]^2], E_H / E_X [nsys] (host, may be NULL), stats_hosts [nsys] host
 * pointers to [Ns[i](Ns[i]+1)/2 + 1] stats each (array or entries may be
 * NULL). Systems are ordered by cost and spread over `lanes` concurrent host
 * threads (<= 0: 4), each lane with its own handle per mesh and its own stream;
 * handles are cached across calls (released by dg_release_cached_handles) and
 * their source-batch size is chosen by the autotuner unless opts->batch > 0.
 * Returns the worst status over the systems. */
int dg_exchange_build_multi(const dg_mesh_desc* meshes, const double* const* psi_devs, const int32_t* Ns,
                            int32_t nsys, const dg_solver_opts* opts, double* const* K_hosts, double* E_H,
                            double* E_X, dg_solve_stats* const* stats_hosts, int32_t lanes, void* cuda_stream);

/* Frees the handles cached by dg_exchange_build_multi. */
void dg_release_cached_handles(void);

/* Autotuner: times the fine-level operator and smoother for source-batch
 * sizes 8..512 (within ~2 GB of vectors) and sets the handle's batch to the
 * smallest size within 10 % of the best time per source (at most
 * max_sources). In the mixed modes, where the fine level's patch solves run
 * on the tensor cores, it then times the tile shapes of that kernel (2, 4, 6,
 * 8 or 10 patches per work item, i.e. MMA widths N of 32-128 columns) at that
 * batch and keeps the fastest; the shape changes no result. Results are
 * cached per GPU name, mesh and precision in $DG_AUTOTUNE_CACHE (default
 * ~/.cache/dgx_autotune.jsonl). *batch receives the batch choice. */
int dg_autotune_batch(dg_handle h, int32_t max_sources, int32_t* batch);

/* Matrix-free SIPDG operator of multigrid level `level` (0 = fine) applied to
 * B fields: out = A u. u_dev, out_dev: [B][Nq_level] device arrays of the
 * handle's working precision for that call: FP64 when fp32 == 0, FP32 when
 * fp32 == 1. Exposed for tests and for timing the operator kernel alone: the
 * call is stream-ordered and returns without synchronising the stream. */
int dg_apply_operator(dg_handle h, int32_t level, int32_t fp32, const void* u_dev, void* out_dev,
                      int64_t B, void* cuda_stream);

/* Grid transfer between multigrid levels `level` and `level` + 1 (Sec. 6.4:
 * GL interpolation from degree p_c to p on the same mesh, or from a degree-1
 * element to its 8 children), applied to B fields. direction 0
 * (prolongation): out = P in, in_dev [B][Nq_(level+1)], out_dev
 * [B][Nq_level]; direction 1 (restriction): out = P^T in, in_dev
 * [B][Nq_level], out_dev [B][Nq_(level+1)]. Device arrays, FP64 (fp32 == 0)
 * or FP32 (fp32 == 1). Exposed for tests and kernel timing; stream-ordered,
 * no synchronisation. DG_ERR_INVALID_ARG unless 0 <= level < levels - 1. */
int dg_apply_transfer(dg_handle h, int32_t level, int32_t direction, int32_t fp32, const void* in_dev,
                      void* out_dev, int64_t B, void* cuda_stream);

/* Preconditioner of the multigrid smoother of level `level` applied to B
 * fields: z = M r with M the additive Schwarz operator sum_P R_P^T A_P^-1 R_P
 * (DG_SMOOTH_SCHWARZ) or D^-1 (DG_SMOOTH_JACOBI); on the coarsest level M is
 * the exact inverse A_c^-1. r_dev, z_dev: [B][Nq_level] device arrays, FP64
 * (fp32 == 0) or FP32 (fp32 == 1). Exposed for tests and kernel timing; the
 * call is stream-ordered and returns without synchronising the stream. */
int dg_apply_smoother(dg_handle h, int32_t level, int32_t fp32, const void* r_dev, void* z_dev, int64_t B,
                      void* cuda_stream);

/* The patch solves of the Schwarz smoother on level `level` alone (Sec. 3.4:
 * each element patch problem solved exactly by fast diagonalisation), without
 * the gather that sums them: zp[b][e][(p+3)^3] = A_P(e)^-1 R_P(e) r_b, patch
 * node (i, j, k) at i + (p+3)(j + (p+3)k), entries outside the domain 0.
 * FP32 calls on a handle whose level uses the tensor-core kernel run that
 * kernel. r_dev: [B][Nq_level]; zp_dev: [B][E_level][(p_level+3)^3]; device
 * arrays, FP64 (fp32 == 0) or FP32 (fp32 == 1); B <= 65535; level below the
 * coarsest. Exposed for tests and for timing the patch-solve kernel alone;
 * stream-ordered, returns without synchronising. DG_ERR_UNSUPPORTED for a
 * Jacobi handle. */
int dg_apply_patch_solves(dg_handle h, int32_t level, int32_t fp32, const void* r_dev, void* zp_dev, int64_t B,
                          void* cuda_stream);

/* Same result as dg_apply_smoother, for callers that cannot allocate device
 * memory at call time: code running where cudaMalloc is forbidden or would
 * break a memory budget fixed in advance (a pool-managed serving process, a
 * real-time loop, a host that owns every allocation itself). The paper has no
 * counterpart; this is a library-interface variant.
 *
 * This call allocates nothing: the patch scratch is a static device array of
 * 8 MiB (1,048,576 doubles or 2,097,152 floats) and the source list a static
 * array of 256 ints, held by every GPU that loads this library until the
 * process exits. Limits: B <= 256 and B * E_level * (p_level + 3)^3 <= the
 * scratch in the chosen precision (E_level, p_level: elements and degree of
 * the level); larger requests return DG_ERR_INVALID_ARG with a message in
 * dg_last_error_detail. Supported: DG_SMOOTH_SCHWARZ levels and the coarsest
 * level (its exact inverse); a Jacobi handle returns DG_ERR_UNSUPPORTED.
 * The handle itself comes from dg_poisson_setup, which does allocate.
 *
 * The first call on each device looks the static arrays up
 * (cudaGetSymbolAddress) and writes the source list once (a synchronous
 * copy), with that device current. That set-up holds the library's
 * device-wide lock, so the graph captures of the library's own multi-system
 * build are not disturbed by it; a capture the caller runs is invisible to
 * the library: make that first call before any stream capture of the
 * caller's. Every call shares
 * the scratch and overwrites it (nothing in it has to start at zero); calls
 * that overlap on the GPU, on any stream or handle, race on it. Stream-ordered;
 * returns without synchronising the stream. r_dev, z_dev: [B][Nq_level] device
 * arrays, FP64 (fp32 == 0) or FP32 (fp32 == 1). */
int dg_apply_smoother_noalloc(dg_handle h, int32_t level, int32_t fp32, const void* r_dev, void* z_dev, int64_t B,
                              void* cuda_stream);

/* Right-hand side of the pair solves for B sources (steps S1-S4: Sec. 6.1.2
 * and Sec. 6.3): b = 4 pi W f + the Nitsche load of the source's Coulomb
 * boundary data g(f), i.e. sum over boundary faces of int g (sigma v -
 * d_n v) against every test function v, exactly as the solves form it (the
 * handle's boundary route and, in the mixed modes, the FP32 Gaussian-sum
 * tables). f_dev, b_dev: [B][Nq] device FP64. Exposed for tests; returns after
 * synchronising the stream. */
int dg_form_rhs(dg_handle h, const double* f_dev, int64_t B, double* b_dev, void* cuda_stream);

/* Boundary data g of Sec. 6.3 for B sources f_dev [B][Nq] (device): g_dev
 * [B][n_face_nodes] (device, FP64; the Gaussian-sum route is evaluated in FP32
 * with a 1e-7 table when the handle is in a mixed mode, as in the solves), faces in the order -x,+x,-y,+y,-z,+z, each
 * face a 2-D grid of its two tangential global node indices with the lower
 * axis fastest. route: DG_BC_*. Returns the total face-node count in
 * *n_face_nodes when g_dev is NULL. */
int dg_boundary_data(dg_handle h, int32_t route, const double* f_dev, int64_t B, double* g_dev,
                     int64_t* n_face_nodes, void* cuda_stream);

/* Number of CUDA kernels this library has launched in the calling process
 * since it was loaded (all handles, all streams). For profiling and for
 * benchmarks that report how many of the library's kernels ran. */
/* The Gaussian-sum approximation of 1/r that the setup builds for the
 * boundary data (Sec. 6.3, Gaussian-sum approximation): accurate to relative
 * tolerance tol on the distances [rmin, rmax], by the construction
 * `construction` (as dg_solver_opts.gauss_construction: 0 tabulated short sum
 * with the trapezoidal rule as fallback, 1 trapezoidal rule). Host only; needs
 * no GPU. n_terms (host) receives its length and relerr (host, may be NULL) its
 * measured max relative error on 3000 log-spaced distances; c_host and
 * alpha_host (host, [max_terms], may be NULL) receive the coefficients and
 * exponents of 1/r ~ sum_k c_k exp(-alpha_k r^2). DG_ERR_INVALID_ARG for
 * rmin <= 0, rmax <= rmin, tol <= 0, a construction other than 0 or 1, or
 * max_terms smaller than the sum when c_host or alpha_host is given;
 * DG_ERR_UNSUPPORTED when no sum meets tol. */
int dg_gauss_sum(double rmin, double rmax, double tol, int32_t construction, int32_t max_terms, int32_t* n_terms,
                 double* relerr, double* c_host, double* alpha_host);

/* Density callback of the octree refinement: out[i] = rho(xyz[3 i], xyz[3 i + 1],
 * xyz[3 i + 2]) for i < n (host arrays); user is passed through. */
typedef void (*dg_density_fn)(const double* xyz, int64_t n, double* out, void* user);

/* Adaptive octree auxiliary mesh (Sec. 6.2), host side: the uniform root grid
 * `root` (box, n per axis, degree p) refined by 8-child splits of every leaf
 * whose indicator Q = |I_K(rho) - sum over its children of I_C(rho)| (degree-p
 * tensor Gauss-Legendre rules) exceeds delta, while its level is below
 * max_level, and kept 2:1 balanced across faces; repeated until no leaf is
 * split. leaves_host: [max_leaves][4] (host, may be NULL to query the count)
 * receives (level, ix, iy, iz) of every leaf, the leaf occupying
 * [lo + i h_level, lo + (i + 1) h_level] with h_level = (hi - lo) / (n 2^level),
 * in element order (root cell x-fastest, then level, z, y, x); n_leaves (host)
 * the count. Host only; needs no GPU. DG_ERR_INVALID_ARG for a bad root mesh,
 * delta <= 0, max_level outside 0..20, a NULL rho, or max_leaves below the
 * count when leaves_host is given; DG_ERR_NO_MEMORY beyond 2^24 leaves. The
 * operator and the solver on this mesh: dg_octree_apply, dg_octree_setup. */
int dg_octree_refine(const dg_mesh_desc* root, double delta, int32_t max_level, dg_density_fn rho, void* user,
                     int32_t max_leaves, int32_t* leaves_host, int32_t* n_leaves);

/* Face connectivity of a 2:1 balanced set of octree leaves over `root` (as
 * dg_octree_refine returns them; leaves_host [n_leaves][4], host). For leaf e
 * and face f = 2 d + s (s = 1 for the +d face), entry o = 6 e + f:
 *   kind_host[o]: 0 boundary, 1 same-size neighbour, 2 larger neighbour (this
 *     face is a quarter of its face), 3 four smaller neighbours;
 *   nb_host[4 o + j]: the neighbour leaf indices (kinds 1 and 2: j = 0; kind 3:
 *     j = b0 + 2 b1 with b0, b1 the position along the lower and the higher
 *     tangential axis), -1 elsewhere;
 *   pos_host[o]: for kind 2 the quarter of the larger face, b0 + 2 b1 as
 *     above, else -1.
 * Host arrays, written. Host only; needs no GPU. DG_ERR_INVALID_ARG for a bad
 * root mesh, leaves outside the root grid or repeated, or a set that is not a
 * 2:1 balanced partition along some face. */
int dg_octree_faces(const dg_mesh_desc* root, const int32_t* leaves_host, int32_t n_leaves, int32_t* kind_host,
                    int32_t* nb_host, int32_t* pos_host);

/* SIPDG operator on octree leaves (Sec. 3.4 eq. sip_bilinear with symmetric
 * Nitsche boundary terms; Sec. 6.2 mesh): out = A u for B fields, matrix-free
 * on the GPU. Faces between leaves of different size are integrated on the
 * quarters of the larger face; the penalty (p+1)^2/(eps h) (penalty_form 0) or
 * (p+1)^2/(eps h^2) (1) uses the smaller leaf. root, leaves_host [n_leaves][4]
 * (host): a 2:1 balanced leaf set as from dg_octree_refine; u_dev, out_dev
 * [B][n_leaves][(p+1)^3] device FP64, element-blocked in leaf order, nodes
 * x-fastest. Builds its connectivity and tables per call (device memory
 * allocated and freed inside) and synchronises the stream before it returns.
 * u_dev and out_dev must not overlap (out is written while other blocks still
 * read u): overlapping buffers return DG_ERR_INVALID_ARG. The function takes
 * no array lengths: the caller guarantees both hold B * n_leaves * (p+1)^3
 * doubles. DG_ERR_INVALID_ARG for a bad mesh or leaf set (a leaf lying inside
 * another leaf of the set included), penalty arguments, or B outside
 * 0..65535. */
int dg_octree_apply(const dg_mesh_desc* root, const int32_t* leaves_host, int32_t n_leaves, int32_t penalty_form,
                    double penalty_eps, const double* u_dev, double* out_dev, int64_t B, void* cuda_stream);

/* Poisson solver on the octree auxiliary mesh (Sec. 6.2 mesh, Sec. 6.3 boundary
 * data, Sec. 6.1.2 exchange build). The handle keeps the leaves' connectivity,
 * node coordinates, quadrature weights and preconditioner tables on the
 * device; the system is the one dg_octree_apply applies (SIPDG, symmetric
 * Nitsche boundary terms, hanging faces on the smaller face, penalty of the
 * smaller leaf). Every leaf's diagonal block is inverted exactly by fast
 * diagonalisation (the block is a Kronecker sum of 1-D leaf matrices and GL
 * masses): the leaf-block preconditioner P. Dirichlet data: the
 * direct quadrature g(x) = sum_q W_q f(q) / |x - x_q| over all nodes at the GL
 * nodes of every boundary face (Sec. 6.3), imposed weakly by the Nitsche load
 * int_F g (sigma v - d_n v). Solved in FP64 by PCG (preconditioner below).
 *
 * dg_octree_setup: root, leaves_host [n_leaves][4] (host) as for
 * dg_octree_apply; penalty_form / penalty_eps as there; rtol: FP64 true
 * relative residual ||b - A v|| / ||b|| at which a solve stops (0 < rtol < 1);
 * max_iter: PCG iteration limit (>= 1); precond: 1 (default) an hp-multigrid
 * V-cycle, 0 the leaf-block inverse alone. The V-cycle (Sec. 6.4: degree
 * coarsening, then the nested h-hierarchy) smooths each octree level by
 * Chebyshev(3) on P^-1 A (P the leaf-block inverse, lambda_max(P^-1 A) by
 * power iteration at set-up), coarsens the degree per leaf p -> max(1, p/2)
 * down to 1, then restricts to the uniform root grid at degree 1 (every leaf
 * lies in one root cell, so the root space is nested) and applies that grid's
 * own multigrid V-cycle (a uniform solver handle, h-coarsening and a dense
 * coarsest solve). precision: DG_PREC_FP64 (PCG, V-cycle and operator in
 * FP64) or DG_PREC_MIXED (the PCG and its V-cycle in FP32 inside FP64
 * iterative refinement: each round solves A e = r for the FP64 residual r to a
 * reduction of 1e-4, adds e in FP64 and recomputes r in FP64, until r meets
 * rtol; right-hand side, residuals and results stay FP64; the boundary data
 * is one 3xTF32 tensor-core GEMM per chunk of sources against the FP32 kernel
 * matrix 1/|xb_j - x_q| that the handle computes once and keeps on the device
 * when it takes at most 48 GB (nodes x boundary face nodes x 4 bytes; else the
 * FP64 direct sum), accurate to about 1e-7 of sum |W f| / r; stats report the
 * inner iterations and the rounds). Writes the handle to *out (NULL on
 * failure). Fields are [.][Nq] FP64 with Nq = n_leaves (p+1)^3, element-blocked
 * in leaf order, nodes x-fastest. DG_ERR_INVALID_ARG for a bad mesh, leaf set
 * or argument; DG_ERR_UNSUPPORTED beyond 2^31 nodes; DG_ERR_NO_MEMORY,
 * DG_ERR_CUDA. Release with dg_octree_destroy (NULL is ignored). Calls on one
 * handle must not overlap; each synchronises its stream before it returns. */
typedef struct dg_oct* dg_oct_handle;
int dg_octree_setup(const dg_mesh_desc* root, const int32_t* leaves_host, int32_t n_leaves, int32_t penalty_form,
                    double penalty_eps, double rtol, int32_t max_iter, int32_t precond, int32_t precision,
                    dg_oct_handle* out);
void dg_octree_destroy(dg_oct_handle h);
/* Text of the last CUDA failure on the handle ("" if none). */
const char* dg_octree_error_detail(dg_oct_handle h);

/* Node coordinates xyz_dev [Nq][3] and quadrature weights w_dev [Nq] (device,
 * written; either may be NULL, not both). W_q = w_a w_b w_c h_x h_y h_z / 8. */
int dg_octree_node_coords(dg_oct_handle h, double* xyz_dev, double* w_dev, void* cuda_stream);

/* The operator on the handle's mesh: out = A u for B fields (0..65535), u_dev
 * and out_dev [B][Nq] device, not overlapping (DG_ERR_INVALID_ARG). Stream
 * ordered: launches one kernel and returns without synchronising. */
int dg_octree_operator(dg_oct_handle h, const double* u_dev, double* out_dev, int64_t B, void* cuda_stream);

/* The handle's preconditioner alone for B fields: z = V(r), one V-cycle
 * (precond 1), or z = P r, the exact inverse of A's leaf blocks (precond 0).
 * r_dev, z_dev [B][Nq] device, not overlapping. Synchronises the stream. */
int dg_octree_precond(dg_oct_handle h, const double* r_dev, double* z_dev, int64_t B, void* cuda_stream);

/* Solves -Lap v = 4 pi f with the Coulomb boundary data of f for B sources
 * f_dev [B][Nq] (device, read). v_dev [B][Nq] (device, written; may be NULL),
 * stats_host [B] (host, may be NULL): iterations, status, final FP64 true
 * relative residual, self-energy (f|f) = sum_q W_q f v. Returns DG_OK or the
 * worst per-source status (DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN,
 * DG_ERR_NONFINITE for a source with NaN or infinity, whose v is 0). */
int dg_octree_solve(dg_oct_handle h, const double* f_dev, int64_t B, double* v_dev, dg_solve_stats* stats_host,
                    void* cuda_stream);

/* Exchange build on the octree (as dg_exchange_build): the Hartree solve for
 * rho = sum_k psi_k^2, the N(N+1)/2 pair solves f = psi_i psi_j (i <= j), the
 * accumulation W_j = sum_s psi_s v_sj, K = Psi^T diag(W_q) W (K_host [N*N]
 * row-major, host), E_H = (rho|rho) / 2 and E_X = -tr K / 2 (host, may be
 * NULL). psi_dev [N][Nq] device; stats_host [N(N+1)/2 + 1] (host, may be
 * NULL), entry 0 the Hartree solve. N in 1..4096. Returns as dg_octree_solve. */
int dg_octree_exchange_build(dg_oct_handle h, const double* psi_dev, int32_t N, double* K_host, double* E_H,
                             double* E_X, dg_solve_stats* stats_host, void* cuda_stream);

/* Exercises the bounded wait used by every tensor-core kernel of this library
 * (their pipeline hand-offs are mbarrier waits that give up after about a
 * second and report DG_ERR_TIMEOUT instead of hanging): one warp waits on an
 * mbarrier that it arrives on (arrive != 0) or that nothing ever arrives on
 * (arrive == 0), for at most limit_cycles SM clock cycles (1 .. 2^34). Returns
 * DG_OK when the wait completed, DG_ERR_TIMEOUT when it gave up (the CUDA
 * context stays usable), DG_ERR_INVALID_ARG for a limit out of range. The
 * paper has no counterpart: this is a test hook for the failure path.
 * Synchronises the stream; allocates and frees one int. */
int dg_wait_probe(int32_t arrive, int64_t limit_cycles, void* cuda_stream);

int64_t dg_kernel_launch_count(void);

/* Releases the handle and all device memory it owns. NULL is ignored. */
void dg_destroy(dg_handle h);

/* Static text for a DG_* code. */
const char* dg_error_string(int status);

/* Message describing the last failure on h (empty string if none). */
const char* dg_last_error_detail(dg_handle h);

#ifdef __cplusplus
}
#endif

#endif /* DG_POISSON_H */
