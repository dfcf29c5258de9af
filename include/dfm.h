/*
 * dfm.h -- C ABI of the GB300 discrete-flow-mapping library (libdfm.so).
 *
 * Discrete flow mapping (DFM) transports a phase-space boundary density
 * through a conforming tetrahedral mesh.  The library implements the
 * data-parallel hot path of the method of Bajars, Chappell, Sondergaard and
 * Tanner ("Transport of phase space densities through tetrahedral meshes
 * using discrete flow mapping"):
 *
 *   1. assembly of the Galerkin matrix B of the weighted boundary transfer
 *      operator (Sec. 3.2, Eqs. Bapprox and B4DInt): for every tetrahedron and
 *      every ordered pair (l, l') of its faces an N_b x N_b block, with the
 *      spatial integral done in closed form (Sec. 3.3) and the direction
 *      integral by quadrature over the seven direction sub-regions (Sec. 3.4);
 *   2. the stationary solve (I - B) rho = rho0 (Sec. 2, Eqs. NSum/GovIE);
 *   3. the interior density functional (Sec. 4.1, Eq. IntDens) and the adjoint
 *      gradient of a receiver functional with respect to per-tet damping.
 *
 * Conventions shared by every entry point:
 *   - tet t has vertices (v0, v1, v2, v3); face f is the face opposite v_f,
 *     with vertices (v_{f+1}, v_{f+2}, v_{f+3}) (indices mod 4); it is row
 *     r = 4 t + f of every coefficient vector;
 *   - the face frame (the paper leaves it open, Sec. 3.3): origin at the
 *     first face vertex, e1 along the first edge, n the inward unit normal
 *     (towards v_f), e2 = n x e1; the tangential momentum of an inward unit
 *     direction d is p = (d.e1, d.e2);
 *   - momentum basis: Zernike polynomials Z_n^m, n = 0..Np, m = -n, -n+2, .., n
 *     (Sec. 3.1), index (n (n+2) + m) / 2, N_b = (Np+1)(Np+2)/2;
 *   - a coefficient vector is rho[row][N_b] (row-major, FP64 unless stated);
 *     R right-hand sides are stored one after the other: rho[R][rows][N_b];
 *   - uniform media (c = rho_f = 1): a ray leaving through an interior face is
 *     transmitted with probability 1 into the neighbour (Sec. 3.3 with equal
 *     impedances); at a boundary face it is specularly reflected with weight
 *     r (the face's reflection coefficient; r = 0 is an open boundary).
 *
 * Memory: mesh arrays passed to dfm_mesh_create are HOST pointers and are
 * copied.  Every other array argument is a DEVICE pointer owned by the caller
 * unless stated.  Handles (dfm_mesh, dfm_op) are owned by the library and
 * freed by their destroy call.  Work runs on the CUDA stream given
 * (a cudaStream_t passed as void*, NULL = legacy default stream); calls
 * return after enqueueing except where a result must come back to the host
 * (stated per call).
 *
 * Errors: every int-returning call returns DFM_OK (0) or a negative DFM_ERR_*
 * code and never throws; dfm_last_error() returns a message for the calling
 * thread's last failure.
 */
#ifndef DFM_H
#define DFM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DFM_OK 0
#define DFM_ERR_ARG (-1)           /* invalid argument (NULL, size, range) */
#define DFM_ERR_MESH (-2)          /* degenerate tet, non-manifold face, bad index */
#define DFM_ERR_CUDA (-3)          /* a CUDA runtime call failed */
#define DFM_ERR_OOM (-4)           /* device allocation failed */
#define DFM_ERR_NOT_CONVERGED (-5) /* iteration cap reached; info still filled */
#define DFM_ERR_NONFINITE (-6)     /* NaN/Inf met in a residual or input */
#define DFM_ERR_UNSUPPORTED (-7)   /* option combination not built */

/* storage/arithmetic precision of operator blocks */
#define DFM_F64 0
#define DFM_F32 1
#define DFM_BF16 2
#define DFM_F16 3
#define DFM_FP8E4M3 4 /* preconditioner copy only: e4m3 values with one FP32 scale per operator row */

/* Basis codes.  Every argument named Np takes the momentum order N_p in its
 * low 8 bits and the spatial basis on each face in the bits above:
 * DFM_BASIS(Np, 0) = Np is the paper's piecewise-constant function per face
 * (Sec. 3.1), N_b = (Np+1)(Np+2)/2 unknowns per face (row); DFM_BASIS(Np, 1)
 * is the linear basis, the finer spatial approximation Sec. 3.1 and the end
 * of Sec. 4.1 point to: three orthonormal affine functions per face, from
 * Gram-Schmidt of (1, l_1, l_2) with l_k the barycentric coordinate of the
 * face's k-th vertex in frame order (the vertex order of the face frame),
 * 3 N_b unknowns per row ordered s N_b + (Zernike index), s = 0 the constant.
 * The linear basis is built for Np <= 8, FP32 blocks, uniform media, moment 0,
 * without the adjoint contraction and point sources. */
#define DFM_BASIS(Np, s) ((Np) | ((s) << 8))

/* stationary solvers */
#define DFM_SOLVE_NEUMANN 0   /* x <- rho0 + B x (Eq. NSum), FP64 */
#define DFM_SOLVE_GMRES 1     /* restarted GMRES on (I - B) x = rho0 in the operator's precision */
#define DFM_SOLVE_GMRES_IR 2  /* FP64-residual iterative refinement around FP32 GMRES */

typedef struct dfm_mesh dfm_mesh;
typedef struct dfm_op dfm_op;

typedef struct {
  int64_t n_verts;
  int64_t n_tets;
  int64_t n_rows;           /* 4 n_tets */
  int64_t n_boundary_rows;  /* faces on the mesh boundary */
  double min_abs_volume;    /* smallest |tet volume| */
  double total_volume;
} dfm_mesh_info_t;

/* Build a mesh (Sec. 2: conforming tet mesh, per-face neighbours).
 *   verts [n_verts][3] FP64, tets [n_tets][4] int32 (any orientation): HOST.
 *   refl  [4 n_tets] FP64 per-row reflection coefficient in [0, 1] (only
 *         boundary rows are read) or NULL to use refl_default everywhere.
 * Runs the face-matching (open-addressing hash on sorted vertex triples) and
 * face-geometry kernels, then waits on the stream for the mesh check.
 * Errors: DFM_ERR_ARG (sizes, NULL, refl outside [0,1]), DFM_ERR_MESH
 * (vertex index out of range, zero-volume tet, a face shared by > 2 tets). */
int dfm_mesh_create(const double* verts, int64_t n_verts, const int32_t* tets, int64_t n_tets, const double* refl,
                    double refl_default, void* stream, dfm_mesh** out);
void dfm_mesh_destroy(dfm_mesh* mesh);
int dfm_mesh_info(const dfm_mesh* mesh, dfm_mesh_info_t* info);

/* Copy the face matching to the host: recv[4 n_tets] int32, recv[4t+f] = the
 * row that receives flux leaving tet t through face f (the neighbour's row, or
 * 4t+f itself on the boundary).  Blocks until copied. */
int dfm_mesh_recv(const dfm_mesh* mesh, int32_t* recv_host);

/* Face matching (the recv map of dfm_mesh_recv) WITHOUT ANY DEVICE ALLOCATION.
 * The paper has no counterpart: this is a library service for callers that
 * cannot call cudaMalloc -- applications that hand all device memory to their
 * own pool or arena up front (an untracked allocation would fail or fragment
 * it) and code that must not enter the CUDA allocator where it runs.
 *   tets:  device int32 [n_tets][4] (caller-owned input);
 *   recv:  device int32 [4 n_tets] (caller-owned output), same meaning as
 *          dfm_mesh_recv;
 *   n_boundary: host int64, receives the number of boundary rows (or NULL).
 * The hash table lives in a fixed file-scope __device__ array of 2^20 slots
 * (16 MiB), present on every GPU that loads the library until the process
 * exits; meshes above 131,072 tets (or 2^21 - 1 vertices) are rejected with
 * DFM_ERR_ARG.  The first call on a device looks up the array's device
 * address there (cudaGetSymbolAddress); make that first call before any
 * stream capture.  Every call shares the array and re-initialises it, so calls
 * whose work overlaps on the GPU (other streams or host threads on the same
 * device) race and must be serialised by the caller.  Waits on the stream to
 * read back the error flags and the boundary count.  Errors: DFM_ERR_ARG,
 * DFM_ERR_MESH (as dfm_mesh_create), DFM_ERR_CUDA. */
int dfm_face_match_static(const int32_t* tets, int64_t n_verts, int64_t n_tets, int32_t* recv, int64_t* n_boundary,
                          void* stream);

/* Gauss-Legendre nodes and weights on [-1, 1] (the per-patch direction rule,
 * Sec. 3.4), computed on the device in FP64 by Newton iteration on the
 * Legendre three-term recurrence.  x, w: device FP64 [q], 1 <= q <= 64. */
int dfm_gauss_legendre(int q, double* x, double* w, void* stream);

typedef struct {
  int Np;               /* momentum order 0..20 (N_b = (Np+1)(Np+2)/2); above 8 (the orders of the
                           cuboid verification, Sec. 4.1) DFM_F32 blocks only, built by the kernels
                           for wide bases, and applied without preconditioner copies */
  const double* mu;     /* device FP64 [n_tets] damping per tet, or NULL */
  double mu_uniform;    /* damping when mu == NULL (>= 0) */
  int quad_order;       /* Gauss-Legendre order per direction patch; 0 = Np + 6 */
  double max_patch_deg; /* split direction patches until every edge <= this angle; 0 = 60 */
  int precision;        /* DFM_F64 or DFM_F32 (FP32 arithmetic, FP64 geometry set-up) */
  int moment;           /* 0: B itself.  k = 1..3: the k-th damping derivative d^k B / d mu^k at the
                           given damping (every tet's mu moved together), i.e. the spatial factor
                           2|OBC| phi2(mu L_O) replaced by 2|OBC| L_O^k phi2^(k)(mu L_O).  Then
                           B(mu_c + e) = sum_k e^k/k! B^(k): Taylor moments that let right-hand
                           sides with different uniform damping share one set of operators. */
  const double* c;      /* device FP64 [n_tets] propagation speed per tet, or NULL (all 1) */
  const double* rho_f;  /* device FP64 [n_tets] fluid density per tet, or NULL (all 1).  With
                           either given, an interior face between tets of different impedance
                           z = rho_f c or speed is an interface (Sec. 3.3): a ray crossing it is
                           transmitted with probability
                             lambda_t = 4 z_i z_j cos(th_r) cos(th_t) / (z_i cos(th_r) + z_j cos(th_t))^2
                           (Snell: sin(th_t) = (c_i/c_j) sin(th_r); zero beyond the critical angle),
                           its receiving momentum scaled by c_i/c_j, and reflected specularly back
                           into its tet with 1 - lambda_t.  The reflected blocks form a second
                           part of the operator (up to six blocks per row in all), applied with
                           the first by dfm_apply and the solvers; preconditioner copies hold
                           the first part only.  Not with moment > 0 or combined operators. */
} dfm_params;

typedef struct {
  int Np, nb;
  int precision;
  int64_t n_rows;
  int64_t row_stride;   /* elements between consecutive rows of vals */
  const void* vals;     /* device: vals[row][3][nb][nb] (+ padding to row_stride) */
  int64_t bytes;        /* bytes of vals */
} dfm_op_info_t;

/* Assemble B (Sec. 3.2-3.4).  Block layout: row R holds the three blocks
 * that R receives, all from one tet t (t = recv[R]/4, exit face l' =
 * recv[R]%4): slot k is source face l = the k-th face of t other than l'
 * (ascending).  Each block is nb x nb row-major: row = test index (n',m') on
 * the receiving face, column = trial index (n,m) on the source face:
 *   B = lambda N_{n'm'} / sqrt(|T_l||T_l'|) sum_nodes w J S(d) Z_{n'm'}(p') Z_nm(p),
 *   S(d) = 2 A_nabla(d) phi2(mu L_O(d)), phi2(x) = (x - 1 + e^-x)/x^2 (Sec. 3.3).
 * Asynchronous on the stream.  Errors: DFM_ERR_ARG, DFM_ERR_OOM. */
int dfm_assemble(const dfm_mesh* mesh, const dfm_params* params, void* stream, dfm_op** out);
/* Re-assemble into an existing operator of the same mesh, Np and precision
 * (no allocation); used for repeated assembly with new damping. */
int dfm_assemble_into(const dfm_mesh* mesh, const dfm_params* params, dfm_op* op, void* stream);
void dfm_op_destroy(dfm_op* op);
int dfm_op_info(const dfm_op* op, dfm_op_info_t* info);
/* Copy the block storage (dfm_op_info_t.bytes bytes, layout above) to dst, a
 * device or host pointer; asynchronous on the stream. */
int dfm_op_copy_vals(const dfm_op* op, void* dst, int64_t bytes, void* stream);
/* The reflected part of an operator assembled with heterogeneous media
 * (dfm_params.c / rho_f): the same layout and size as dfm_op_copy_vals, row
 * R = 4t + l' holding the blocks reflected at face l' of tet t from the tet's
 * other faces (slot k = the k-th face of t other than l'); zero blocks where
 * l' is not an interface.  DFM_ERR_ARG if the operator has no reflected part. */
int dfm_op_copy_reflected(const dfm_op* op, void* dst, int64_t bytes, void* stream);

/* y = x0 + alpha * B x (trans = 0) or y = x0 + alpha * B^T x (trans = 1) for
 * R right-hand sides; x, y, x0 device [R][rows][nb] of type xtype
 * (DFM_F64 or DFM_F32); x0 may be NULL (treated as 0) or alias x; y must not
 * alias x.  Asynchronous. */
int dfm_apply(const dfm_op* op, const void* x, const void* x0, void* y, int R, double alpha, int trans, int xtype,
              void* stream);

/* Several operators applied together, with per-right-hand-side weights:
 *   y_r = x0_r + alpha * sum_k coef_host[r * K + k] B_k x_r,  r < R, k < K <= 4.
 * ops: K FP32 operators of the same mesh and Np (e.g. the damping moments
 * B^(k) of dfm_params.moment, with coef = (mu_r - mu_c)^k / k!); x, x0, y as
 * for dfm_apply (forward only).  Every operator tile is streamed once per pass
 * over up to 16 right-hand sides.  Asynchronous. */
int dfm_apply_combo(const dfm_op* const* ops, int K, const double* coef_host, const void* x, const void* x0, void* y,
                    int R, double alpha, int xtype, void* stream);

/* Galerkin coefficients of unit isotropic sources (Sec. 3.1-3.2): for source
 * s, rho0[s][row_s][(0,0)] = sqrt(|T_row_s|) and zero elsewhere.
 * rows_host: HOST int64 [n_src] boundary (or any) rows; rho0: device FP64
 * [n_src][rows][nb] (fully overwritten).  Asynchronous. */
int dfm_source(const dfm_mesh* mesh, int Np, const int64_t* rows_host, int n_src, double* rho0, void* stream);

/* Galerkin coefficients of unit boundary densities with one ray direction
 * (Sec. 4.1, Eq. RhoNeumann, generalised from the normal to any inward d):
 * the density delta(p - p_d) on face T_row, p_d = (d.e1, d.e2) the
 * tangential momentum of the unit inward direction d, projects onto
 *   rho0[row][(n,m)] = N_nm Z_n^m(p_d) sqrt(|T_row|),   N_nm = (2n+2)/(eps_m pi)
 * (the inverse norm of Z_n^m on the unit disc, eps_0 = 2, eps_m = 1 else).
 * For d = the inward normal (p_d = 0) only m = 0, n even survive:
 * (n+1)/pi (-1)^(n/2) sqrt(|T_row|).
 *   rows_host: HOST int64 [n_src] rows.  dirs_host: HOST FP64 [n_src][3]
 *   directions (any length > 0; normalised here) or NULL for each row's
 *   inward normal.  combine = 0: rho0 device FP64 [n_src][rows][nb], source s
 *   alone in right-hand side s; combine = 1: rho0 device FP64 [rows][nb], all
 *   sources in one right-hand side (rows must then be distinct).  rho0 is
 *   fully overwritten.
 * Asynchronous when dirs_host is NULL; with directions it waits on the stream
 * and returns DFM_ERR_ARG if some d does not point strictly into its tet
 * (d.n <= 0 after normalisation), leaving rho0 with that source's row zero.
 * Errors: DFM_ERR_ARG (NULL, Np outside 0..20, row out of range, zero
 * direction, repeated row with combine = 1). */
int dfm_source_directed(const dfm_mesh* mesh, int Np, const int64_t* rows_host, const double* dirs_host, int n_src,
                        int combine, double* rho0, void* stream);

/* Galerkin coefficients of point sources in uniform media (Sec. 4.2,
 * Eq. SourceRho): rays leave r0 in every direction and enter the next tet
 * through each face F of the tet holding r0 that does not contain r0; the row
 * across F (on the boundary: F's own row, weighted by its reflection
 * coefficient, the reflected direction keeping the tangential components)
 * receives
 *   rho0[rec][(n,m)] = N_nm / sqrt|F| Int_F strength cos(theta) exp(-mu R) / R^2 Z_n^m(p(u)) ds,
 * u = unit(s - r0), R = |s - r0|, theta the angle between u and F's normal,
 * p(u) the tangential part of u in the receiving face's frame, mu the damping
 * of the tet holding r0 and N_nm as in dfm_source_directed (strength =
 * rho_f omega^2 / (16 pi^2 c) for the paper's acoustic source).  A source on
 * a face, an edge or a vertex (barycentric coordinates within 1e-12 of 0)
 * sends from every tet whose closure holds it, through the faces that do not
 * contain it.  Each face integral runs in FP64: nq = 0 (default) the split
 * polar rule of dfm_interior_density with 24 points per direction, nq < 0 that
 * rule with |nq| points (accurate for sources close to a face), nq > 0 the
 * collapsed tensor Gauss-Legendre rule of order nq on the flat triangle.
 *   r0_host: HOST FP64 [n_src][3] positions.  mu: device FP64 [n_tets] or NULL
 *   for mu_uniform.  rho0: device FP64 [n_src][rows][nb], fully overwritten.
 * Waits on the stream (the tets holding each source are found on the device
 * and counted on the host).  Errors: DFM_ERR_ARG (NULL, Np outside 0..8, |nq|
 * outside 2..64, negative mu_uniform, non-finite position or strength; a
 * source outside the mesh, whose rows then stay zero). */
int dfm_point_source(const dfm_mesh* mesh, int Np, const double* r0_host, int n_src, const double* mu,
                     double mu_uniform, double strength, int nq, double* rho0, void* stream);

typedef struct {
  int method;        /* DFM_SOLVE_* */
  double tol;        /* stop when ||rho0 - (I - B) x|| <= tol ||rho0|| (FP64 residual; Neumann: relative increment) */
  int max_iter;      /* cap on operator applications (0 = 20000) */
  int restart;       /* GMRES restart length, <= 256 (0 = 128) */
  int use_x0;        /* 1: rho holds the initial guess on entry */
  double inner_tol;  /* GMRES_IR: floor of the inner FP32 relative tolerance (0 = 1e-6); an inner
                        solve also stops when a restart cycle gains less than 10% */
  int transpose;     /* 1: solve (I - B)^T x = rho0 instead (the adjoint equation) */
  int poly_degree;   /* right preconditioner p(B) = sum_{k<d} B^k, so GMRES runs on I - B^d:
                        GMRES_IR inner solves: 0 = 16 (48 with a low-precision precond_precision);
                        GMRES on an FP64 operator: 0 = none */
  int precond_precision; /* GMRES_IR: 0 = the polynomial preconditioner uses the operator itself;
                        DFM_F16 or DFM_BF16 = its hops use a 16-bit copy of the blocks (made once
                        per assembly, half the bytes per hop); DFM_FP8E4M3 = an 8-bit e4m3 copy
                        with one FP32 scale per row (a quarter of the bytes); a transposed solve
                        uses the same kinds of copy of B^T; the inner solver is flexible
                        GMRES, which tolerates the inexact preconditioner; the Krylov operator
                        I - B and the FP64 residual keep the FP32 blocks */
  int batch;         /* GMRES_IR with R > 1: right-hand sides iterated in lockstep, sharing
                        every operator pass (0 = up to 16, capped so the group's FP32 Krylov
                        basis stays within 24 GiB) */
  int block;         /* GMRES_IR with R > 1 and a low-precision precond_precision: 1 = block
                        flexible GMRES, one Krylov space spanned by the whole group (block
                        Gram-Schmidt with Cholesky QR, each pass repeated once; restart counts
                        block steps, capped at 512 / group size - 1); 0 = each right-hand side
                        in its own Krylov space, in lockstep.  The operator passes are shared
                        either way; the block space needs fewer of them.  Ignored by
                        dfm_solve_combo / dfm_solve_damped (one operator per right-hand side). */
  int coarse;        /* GMRES_IR, right-hand sides solved one at a time, with a low-precision
                        precond_precision: 0 = off; g in 1..4 = two-level preconditioner
                        z = Q v + p~(B)(v - (I - B) Q v), Q = V (V^T (I - B) V)^{-1} V^T, V the
                        isotropic (0,0) density sqrt|T| on each of g^3 spatial aggregates of tets
                        (boxes of the mesh's bounding box, by tet centroid; empty ones dropped),
                        for the slow near-isotropic mode (not in the paper).  (I - B) V is formed
                        once per call (its g^3 applications are counted in iters), so each
                        preconditioner call adds g^3-long dot and update passes, no application.
                        Ignored by batched and block solves and by dfm_solve_combo. */
} dfm_solve_opts;

typedef struct {
  int iters;         /* operator applications used */
  int outer;         /* refinement steps (GMRES_IR) or restarts */
  double resid;      /* final relative residual (FP64) of the worst right-hand side */
} dfm_solve_info;

/* Stationary density rho = (I - B)^{-1} rho0 (Eq. GovIE) for R right-hand
 * sides, rho0 and rho device FP64 [R][rows][nb].  Synchronises with the
 * stream once per iteration to read convergence scalars.  Returns
 * DFM_ERR_NOT_CONVERGED (info filled, rho = last iterate) at the cap and
 * DFM_ERR_NONFINITE if a residual is not finite. */
int dfm_solve(const dfm_op* op, const double* rho0, int R, double* rho, const dfm_solve_opts* opts, void* stream,
              dfm_solve_info* info);

/* dfm_solve for right-hand sides with their own operators
 * B_r = sum_k coef_host[r * K + k] B_k (see dfm_apply_combo): the stationary
 * densities rho_r = (I - B_r)^{-1} rho0_r, batched as in dfm_solve (every
 * operator pass serves a group of right-hand sides).  opts->method must be
 * DFM_SOLVE_GMRES_IR, no transpose.  With opts->precond_precision set, the
 * preconditioner's hops use a low-precision copy of B_0 alone (the same
 * p(B~_0) for every right-hand side; the Krylov operator is each I - B_r).
 * Errors as dfm_solve. */
int dfm_solve_combo(const dfm_op* const* ops, int K, const double* coef_host, const double* rho0, int R, double* rho,
                    const dfm_solve_opts* opts, void* stream, dfm_solve_info* info);

/* Stationary densities for right-hand sides that each have their own uniform
 * damping mu_r (the absorption factor exp(-mu L) of Sec. 2, in the closed
 * form of Sec. 3.3), from the damping moments of one assembly:
 *   rho_r = (I - B(mu_r))^{-1} rho0_r,
 *   B(mu_r) = sum_{k<K} (mu_r - mu_c)^k / k! B^(k),   B^(k) = d^k B / d mu^k at mu_c,
 * with the Taylor weights computed here.  moments[k] is the operator
 * assembled with dfm_params.moment = k; all K (1..4) share the mesh, Np,
 * FP32 precision and one uniform damping mu_c (dfm_params.mu == NULL,
 * mu_uniform = mu_c), which is read from them.  The truncation error of an
 * entry is bounded by (|mu_r - mu_c| L)^K / K! times the entry's size, L the
 * longest chord of its tet.  mu_rhs_host: HOST FP64 [R], each finite and >= 0;
 * rho0, rho: device FP64 [R][rows][nb].  Solved as dfm_solve_combo with these
 * weights (GMRES_IR only, batched; a low-precision preconditioner copy is made
 * from moments[0] = B(mu_c)).  Errors: DFM_ERR_ARG (a moment of the wrong
 * order, a per-tet damping field or different mu_c, a bad mu_r) and those of
 * dfm_solve. */
int dfm_solve_damped(const dfm_op* const* moments, int K, const double* mu_rhs_host, const double* rho0, int R,
                     double* rho, const dfm_solve_opts* opts, void* stream, dfm_solve_info* info);

/* The inexact polynomial preconditioner of the flexible inner solve
 * (dfm_solve_opts.precond_precision), on its own.  The paper gives no
 * solver; this is a building block for callers' own Krylov methods:
 *   z_r = sum_{k<degree} B~^k x_r  (transpose != 0: sum_{k<degree} (B~^T)^k x_r),  r < R,
 * B~ = the FP16 (precision DFM_F16) or BF16 (DFM_BF16) rounding, to nearest,
 * of op's FP32 blocks, or (DFM_FP8E4M3) s_R q with q the e4m3 rounding (to
 * nearest even, saturating) of B/s_R and s_R = (max |entry| of row R) / 448
 * in FP32 (made on first use and again after each assembly),
 * evaluated by Horner's rule z <- x + B~ z with FP32 vectors and FP32
 * accumulation.  op: FP32 operator; x, z: device FP32 [R][rows][nb], 16-byte
 * aligned, z must not alias x; 1 <= degree <= 64; DFM_ERR_UNSUPPORTED for
 * bases above Np = 8.  Uses a scratch of
 * 3 R rows NBP floats (NBP = nb rounded up to 8) taken with cudaMallocAsync
 * on the stream and released in stream order.  Asynchronous. */
int dfm_precond_apply(const dfm_op* op, int precision, int degree, int transpose, const float* x, float* z, int R,
                      void* stream);

/* CUDA graphs of the preconditioner's Horner chains (process-wide switch,
 * default on).  A chain of degree d >= 4 runs the pack of x, d - 1 hops on
 * the low-precision copy, the last into z; the d - 3 hops in between touch
 * only the chain's scratch, so per operator, copy, right-hand-side count,
 * degree and scratch buffers they are the same launches every time.  The
 * first chain of such a shape runs eagerly (the autotuner's timing happens
 * then), the second is captured into a graph (stream capture, relaxed mode)
 * and later ones replay it as one launch; a capture that fails leaves that
 * shape to eager launches.  Results are bit-identical with graphs on or off.
 * Graphs are kept per operator (at most 16 shapes) and freed with it.
 * mode 1: on, 0: off, -1: query.  Returns the state after the call (0 or 1),
 * or DFM_ERR_ARG for another mode. */
int dfm_hop_graphs(int mode);
/* Hop-chain graph replays so far in this process (each counts its d - 3 hops
 * in dfm_launch_count). */
long long dfm_hop_graph_replays(void);

/* Interior density functional (Sec. 4.1, Eq. IntDens, c = 1): for each listed
 * tet e, the coefficients g_e of
 *   rho_T(r_e) = sum_{l, nm} rho_(e,l,nm) g_e[l][nm],
 *   g_e[l][nm] = |T_l|^{-1/2} Int_{T_l} Z_nm(p(s->r_e)) cos(vartheta) exp(-mu_e |r_e - s|) / |r_e - s|^2 ds,
 * at r_e = the tet's centroid, p(s->r) the tangential part of unit(r - s) in
 * face l's frame, and dg_e = d g_e / d mu_e.  Each face integral runs in
 * FP64 with, for nq < 0, the split polar rule with |nq| points per direction:
 * the face is cut at the foot of r_e into three signed triangles, one per
 * edge, integrated in the polar angle seen from r_e and in the azimuth,
 * sampled through the position along the edge with a tangent substitution
 * (each edge cut at the foot of the perpendicular from the foot of r_e;
 * 6 nq^2 nodes), which stays accurate when r_e is close to the face or its
 * foot close to an edge (thin tets); nq = 0 selects that rule with 24 points
 * per direction (the default; within 1e-13 of the largest entry of the
 * adaptive cubature of the integral on the jittered Kuhn meshes tested).
 * nq > 0 selects a collapsed tensor Gauss-Legendre rule of order nq
 * on the flat triangle, which loses digits (percents of the largest density
 * at order 32) when r_e is close to the face.  |nq| in 2..64.
 *   tets_host: HOST int64 [n] tet ids; weights_host: HOST FP64 [n] or NULL (1).
 *   gvec, dgvec: device FP64 [rows][nb]; on return gvec[4e+l] += w_e g_e[l] and
 *   dgvec[4e+l] += w_e dg_e[l] for the listed tets (other rows untouched), so
 *   J(rho) = gvec . rho and dJ/dmu_e (explicit part) = dgvec[4e..4e+3] . rho[4e..4e+3].
 *   mu: device FP64 [n_tets] or NULL for mu_uniform.  Np in 0..20.  Asynchronous. */
int dfm_interior_density(const dfm_mesh* mesh, int Np, const double* mu, double mu_uniform, const int64_t* tets_host,
                         const double* weights_host, int n, int nq, double* gvec, double* dgvec, void* stream);

/* Per-tet values of a tet-local functional:
 *   out[r][e] = sum_{l < 4} sum_{nm} gvec[4e+l][nm] rho_r[4e+l][nm].
 * With gvec from dfm_interior_density over every tet (weights 1), out[r][e]
 * is the interior density rho_T(r_e) of right-hand side r at tet e's centroid
 * (Sec. 4.1, Eq. IntDens).
 *   gvec: device FP64 [rows][nb]; rho: device FP64 [R][rows][nb];
 *   out: device FP64 [R][n_tets] (overwritten).  Asynchronous.
 * Errors: DFM_ERR_ARG (NULL, R < 1, Np outside 0..20). */
int dfm_tet_density(const dfm_mesh* mesh, int Np, const double* gvec, const double* rho, int R, double* out,
                    void* stream);

/* Adjoint gradient of J = sum_r gvec . rho_r with respect to the per-tet damping
 * (the operator's dependence on mu through exp(-mu L), Sec. 2 and Sec. 3.3):
 *   (I - B)^T lambda = gvec  (solved with opts, transpose forced on),
 *   dJ_dmu[r][t] = sum over the 12 face pairs of tet t of lambda_R^T (dB/dmu_t) rho_r,J
 *                  + dgvec[4t..4t+3] . rho_r[4t..4t+3]   (if dgvec != NULL),
 * with dB/dmu from the same quadrature as the assembly and
 * d/dmu [2 A phi2(mu L_O)] = 2 A L_O phi2'(mu L_O); dB/dmu is never stored.
 *   params: the damping the operator was assembled with (mu, Np, quadrature).
 *   rho: device FP64 [R][rows][nb]; gvec, dgvec: device FP64 [rows][nb] (one
 *   functional shared by all R right-hand sides, so one adjoint solve serves all);
 *   lambda_out: device FP64 [rows][nb]; with opts->use_x0 = 1 it holds the
 *   initial guess on entry (e.g. lambda of an earlier call with the same
 *   operator and functional: the refinement then checks its FP64 residual and
 *   stops at once if it meets tol); dJ_dmu: device FP64 [R][n_tets] (overwritten).
 * Synchronises like dfm_solve.  Errors as dfm_solve; DFM_ERR_UNSUPPORTED for
 * operators above Np = 8 (the contraction is built for bases up to 45). */
int dfm_adjoint(const dfm_op* op, const dfm_params* params, const double* rho, int R, const double* gvec,
                const double* dgvec, double* lambda_out, double* dJ_dmu, const dfm_solve_opts* opts, void* stream,
                dfm_solve_info* info);

/* Data-wait time-outs.  The pipelined kernels (operator applications,
 * preconditioner hops) wait on shared-memory barriers for their bulk copies
 * with a bounded number of polls (a few seconds); a wait that runs out sets
 * the operator's device error flag, lets the copies in flight land and ends
 * the kernel, leaving its output incomplete.  dfm_solve, dfm_solve_combo,
 * dfm_solve_damped and dfm_adjoint read the flag after their iterations and
 * return DFM_ERR_TIMEOUT; after dfm_apply, dfm_apply_combo or
 * dfm_precond_apply the caller reads it with dfm_op_check_error.
 *   dfm_op_check_error: waits on the stream, returns DFM_ERR_TIMEOUT if a
 *     kernel of op timed out since the last check (and clears the flag), else
 *     DFM_OK.
 *   dfm_selftest_timeout: runs one kernel whose wait is on a barrier that
 *     nothing completes, with a limit of `polls` polls (1..1000000, each at
 *     most about a microsecond), so that the time-out path sets op's flag
 *     exactly as a stalled copy would; asynchronous.  For tests of callers'
 *     error handling. */
#define DFM_ERR_TIMEOUT (-8) /* a kernel gave up waiting for its data (see dfm_op_check_error) */
int dfm_op_check_error(const dfm_op* op, void* stream);
int dfm_selftest_timeout(const dfm_op* op, int polls, void* stream);

/* Autotuning of launch geometries (the paper has no counterpart; a library
 * service).  The tensor-core preconditioner hops choose their tile rows and
 * pipeline stages per launch shape (basis, copy precision, right-hand sides
 * per launch, transposition, operator rows, device): on the first launch of a
 * shape every candidate geometry is timed on the call's own arguments with
 * CUDA events (the stream is synchronised; nothing is timed while the stream
 * is being captured into a graph, where the default geometry is used) and
 * the fastest is kept for later launches.  Geometry changes no arithmetic:
 * results are identical with tuning on or off.
 *   dfm_autotune(mode): 0 = fixed default geometries, 1 = tune on first use
 *     (the default), 2 = forget the tuned choices and tune again.
 *   dfm_autotune_report(buf, len): writes a JSON list of the tuned shapes
 *     with their chosen geometry and every candidate's time ([rows per tile,
 *     stages, ms]) into buf (len bytes, NUL-terminated, truncated if short);
 *     returns the bytes needed including the NUL. */
int dfm_autotune(int mode);
int64_t dfm_autotune_report(char* buf, int64_t len);

/* Kernel accounting, for benchmarks and profiling.
 *   dfm_launch_count: number of CUDA kernels this library has launched in the
 *     process so far (all kernels, all streams).
 *   dfm_stats_enable(n): from now on record a CUDA event pair, on the stream
 *     the kernel runs on, around every launch (n = 1) or every n-th launch
 *     (n > 1, per kernel) of the kernels below; 0 stops.  Event records cost
 *     GPU time between kernels, so sampling keeps the measured region close
 *     to an uninstrumented run;
 *   dfm_stats_reset: forget the recorded pairs and counts (events are reused);
 *   dfm_kernel_stats: launches of one kernel since the last reset (all of
 *     them while enabled) and their device milliseconds: the sum over the
 *     timed launches scaled by launches / timed launches (waits for the
 *     recorded events). */
#define DFM_KERNEL_COUNT 10
#define DFM_KERNEL_ASSEMBLE 0 /* operator assembly (one warp per face pair) */
#define DFM_KERNEL_SPMV 1     /* y = x0 + alpha B x */
#define DFM_KERNEL_SPMV_T 2   /* y = x0 + alpha B^T x */
#define DFM_KERNEL_DOT 3      /* Krylov multi-dot */
#define DFM_KERNEL_AXPY 4     /* Krylov multi-axpy */
#define DFM_KERNEL_SPMV64 5   /* y = x0 + alpha B x with FP64 vectors (residuals) */
#define DFM_KERNEL_CONTRACT 6 /* fused lambda^T (dB/dmu) rho per tet */
#define DFM_KERNEL_SPMV16 7   /* preconditioner hop on the low-precision copy */
#define DFM_KERNEL_SPMV16_T 8 /* preconditioner hop on the transposed copy (adjoint solves) */
#define DFM_KERNEL_SPMV64_T 9 /* y = x0 + alpha B^T x with FP64 vectors (adjoint residuals) */
long long dfm_launch_count(void);
int dfm_stats_enable(int on);
int dfm_stats_reset(void);
int dfm_kernel_stats(int kernel, int64_t* launches, double* total_ms);

/* Quadrature nodes evaluated by the last assembly into op (all face pairs);
 * waits for that assembly.  The benchmark turns it into counted FLOPs. */
int dfm_op_nodes(const dfm_op* op, int64_t* nodes);

/* Thread-local message for the last failing call ("" if none). */
const char* dfm_last_error(void);

/* Library version string. */
const char* dfm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DFM_H */
