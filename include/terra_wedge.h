/*
 * terra_wedge.h -- C ABI of the GB300 (sm_103a) matrix-free wedge Stokes library.
 *
 * The library applies the low-order W1-iso-W2 / W1 wedge Stokes operator of
 * TERRA-NG (arxiv 2609.21633) on a radially extruded icosahedral shell:
 * the variable-viscosity symmetric-gradient block A (Eq. elemmat, Eq. matfree,
 * Eq. epsq / Eq. localapply), the divergence B and gradient B^T of the saddle
 * matrix [[A, B^T], [B, 0]] (Sec. 7, Eq. block-precond), and their diagonals
 * (Eq. pmass).  The mesh is built as in Sec. 2: ten diamonds of an
 * icosahedral base grid, recursive normalised-midpoint refinement to
 * 2^l x 2^l cells per diamond, uniform radial extrusion through N_r node
 * layers, each hexahedral cell split implicitly into two wedges.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Status: every function returns tn_status; 0 (TN_OK) on success, a negative
 * code otherwise.  tn_last_error() returns a thread-local message describing
 * the last failure.  No C++ exception crosses this interface.
 *
 * Pointers: arguments named *_dev are DEVICE pointers (cudaMalloc / torch
 * CUDA tensors) owned by the caller; arguments named *_host are host
 * pointers.  The library never frees or retains caller pointers beyond the
 * call (stream-ordered work enqueued by the call reads / writes them later on
 * that stream).  The library owns the mesh hierarchy, the per-level
 * viscosity and geometry tables and its workspaces.
 *
 * Streams: every operator call is enqueued on the given cudaStream_t
 * (passed as void*, NULL = legacy default stream) and returns without
 * synchronising, unless stated otherwise.
 *
 * Levels: a mesh holds a hierarchy of nested levels h = 0 (finest, the
 * created lateral level l and N_r node layers) to depth-1; level h+1 has
 * lateral level l_h - 1 and (N_r,h - 1)/2 + 1 node layers.  The pressure
 * space of level h (Sec. 3: W1 on the grid one level coarser) is the node set
 * of level h+1.
 *
 * Node layout (velocity components and scalars) of a level with N = 2^l_h,
 * N_r node layers and row pitch P = round_up(N + 1, 4):
 *     index(d, k, i, j) = ((d * N_r + k) * (N + 1) + i) * P + j
 * d in [0,10) diamond, k in [0,N_r) radial node layer (radius r_k), i, j in
 * [0, N] lattice position; j >= N+1 are padding (never read, never written).
 * A velocity field is three such arrays (structure of arrays, one per
 * Cartesian component x, y, z).  Lattice points on diamond edges exist in
 * every diamond that shares them (2 copies on edges, 3 at the ten non-polar
 * icosahedral vertices, 5 at the poles); inputs must hold equal values on all
 * copies and outputs hold bitwise-equal values on all copies.
 * Diamond corners (c00, c10, c01, c11) = lattice (0,0), (N,0), (0,N), (N,N):
 * north d = k: (N, U_k, U_k+1, L_k); south d = 5 + k: (U_k+1, L_k, L_k+1, S),
 * U_k at latitude +atan(1/2), longitude 72k deg; L_k at -atan(1/2), 36 + 72k deg.
 * Radii r_k = r_in + ((r_out - r_in) * k) / (N_r - 1).
 *
 * Wedge layout (per-wedge viscosity): cell (d, i, j) between node layers k and
 * k+1 (i, j in [0, N), k in [0, N_r - 1)) holds wedge W0 = lateral
 * (i,j),(i+1,j),(i,j+1) and W1 = (i+1,j+1),(i,j+1),(i+1,j):
 *     windex(d, k, i, j, w) = (((d * (N_r - 1) + k) * N + i) * N + j) * 2 + w
 *
 * Boundary conditions: at node layers 0 (r_in) and N_r - 1 (r_out) each node
 * carries a projector P_j = I - s_j s_j^T (free-slip, s_j the unit radial
 * direction) or P_j = 0 (no-slip); elsewhere P_j = I.  The constrained
 * velocity block is P A P + (I - P); B acts as B P and B^T as P B^T.
 */
#ifndef TERRA_WEDGE_H
#define TERRA_WEDGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int tn_status;
enum {
  TN_OK = 0,
  TN_EINVAL = -1,        /* invalid argument (NULL, size, aliasing, level out of range) */
  TN_ENOMEM = -2,        /* device or host allocation failed */
  TN_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed */
  TN_ENOTCONVERGED = -4, /* an iterative solve did not reach its tolerance */
  TN_ETIMEOUT = -5,      /* a bounded device wait ran out */
  TN_EBUSY = -6,         /* resource temporarily unavailable (serving admission) */
  TN_ESTATE = -7,        /* call order violated (e.g. apply before set_viscosity) */
  TN_ECANCELED = -8      /* a serving request was cancelled (tn_server_cancel) */
};

typedef enum { TN_F64 = 0, TN_F32 = 1 } tn_prec;
typedef enum { TN_BC_FREESLIP = 0, TN_BC_NOSLIP = 1 } tn_bc;
/* Storage of the per-wedge viscosity that the FP32 kernels read (the FP64 kernels always read
 * FP64).  TN_ETA_BF16 / TN_ETA_F16 keep 16-bit values eta / c plus one FP32 factor c per radial
 * column of wedges (lateral wedge (d, i, j, w) over all radial cells), c = sqrt(min * max) of the
 * column, so the stored values straddle 1; used on levels with N >= 16, FP32 on coarser ones. */
typedef enum { TN_ETA_F32 = 0, TN_ETA_BF16 = 1, TN_ETA_F16 = 2 } tn_eta_storage;
/* Arithmetic of the FP64 element ops (A with its residual and smoother epilogues, B, B^T and the
 * interior layers of diag(A)) on levels with N >= 32, where it bounds the apply:
 * TN_FP64_ELEM_DOUBLE_FLOAT evaluates them (Eq. epsq / Eq. localapply and the one-point B) in
 * double-float (pairs of FP32 numbers, about 48 significand bits, on the FP32 pipe; each
 * operation's error is below 2^-44 of its operands' magnitude), with binary64 inputs, outputs, boundary projections,
 * interface sums and epilogues; TN_FP64_ELEM_BINARY64 in IEEE binary64 throughout.  Coarser levels
 * and the node-block diagonals always use binary64. */
typedef enum { TN_FP64_ELEM_DOUBLE_FLOAT = 0, TN_FP64_ELEM_BINARY64 = 1 } tn_fp64_element;

typedef struct tn_mesh tn_mesh;

typedef struct {
  int bc_inner;       /* tn_bc at r_in  (default TN_BC_FREESLIP) */
  int bc_outer;       /* tn_bc at r_out (default TN_BC_FREESLIP) */
  int div_term;       /* 1: keep the -2/3 div div term of Eq. elemmat (default); 0: drop it */
  int max_levels;     /* upper bound on the hierarchy depth (0 = as deep as possible) */
  int eta_storage;    /* tn_eta_storage of the FP32 path's viscosity (default TN_ETA_F32) */
  double hg_kappa;    /* hourglass control of the A block, Eq. hgstab (default 0 = off): every level's
                       * element matrices get eps_e sum_m,d (g_m x e_d)(g_m x e_d)^T with
                       * eps_e = hg_kappa tr(A_e) / 18 and g_m the hourglass vectors of Eq. hourglass
                       * minus their physical linear part (rigid motions keep zero energy) */
  int radial_quad_points; /* quadrature of the A block (0 or 1 = default: one point at the wedge
                       * barycentre, Sec. 4; 2: the second radial point, the two-point Gauss rule in
                       * the radial reference coordinate at the lateral barycentre, weights 1/2, one
                       * viscosity per wedge).  B, B^T and the pressure mass keep the one-point rule.
                       * 2 together with hg_kappa > 0 is TN_EINVAL (two remedies of the same modes). */
  int fp64_element;   /* tn_fp64_element (default TN_FP64_ELEM_DOUBLE_FLOAT) */
} tn_mesh_opts;

typedef struct {
  int lateral_level;  /* l_h */
  int N;              /* 2^l_h */
  int n_r;            /* radial node layers */
  int pitch;          /* row pitch P (elements) */
  int64_t layer_stride;    /* (N+1) * P */
  int64_t diamond_stride;  /* N_r * (N+1) * P */
  int64_t n_layout;        /* 10 * diamond_stride: elements of one scalar / component array */
  int64_t n_unique_nodes;  /* (10 N^2 + 2) N_r */
  int64_t n_cells;         /* 10 N^2 (N_r - 1) hexahedral cells */
  int64_t n_wedges;        /* 2 n_cells: elements of a per-wedge array */
  int depth;               /* number of levels in the hierarchy */
  double r_in, r_out;
} tn_level_info;

/* Thread-local message of the last failure on this thread (never NULL). */
const char* tn_last_error(void);

/* Build the mesh hierarchy (Sec. 2) on the current CUDA device.
 * lateral_level >= 1; radial_layers = N_r >= 3 node layers with N_r - 1 even
 * (the pressure space coarsens radially too, Sec. 3); 0 < r_in < r_out.
 * opts may be NULL (defaults).  Synchronous; allocates device tables. */
tn_status tn_mesh_create(int lateral_level, int radial_layers, double r_in, double r_out,
                         const tn_mesh_opts* opts, tn_mesh** out);
tn_status tn_mesh_destroy(tn_mesh* mesh);
tn_status tn_mesh_info(const tn_mesh* mesh, int level, tn_level_info* info);

/* Unit-sphere lattice points of a level, host copy: xyz_host[3 * ((d*(N+1)+i)*(N+1)+j) + c]
 * (10 * (N+1)^2 * 3 doubles).  Synchronous. */
tn_status tn_mesh_lateral_points(const tn_mesh* mesh, int level, double* xyz_host);

/* Canonical copy of every layout node of a level, host copy (n_layout int64):
 * canon[index(d,k,i,j)] = smallest layout index holding the same physical node;
 * -1 on padding.  Lets callers build inputs that are equal on all copies. */
tn_status tn_mesh_canonical_index(const tn_mesh* mesh, int level, int64_t* canon_host);

/* Per-wedge viscosity of level 0 (wedge layout, n_wedges doubles, eta > 0),
 * one value per wedge evaluated at the quadrature point q_c (Sec. 4).
 * Copied into the library; coarser levels get the mean of their 8 child
 * wedges.  Stream-ordered. */
tn_status tn_set_viscosity(tn_mesh* mesh, const double* eta_wedge_dev, void* stream);

/* Viscosity law of tn_set_temperature: eta_e = (jump_factor if r_mid < jump_r else 1)
 * * exp(E * (1/2 - T(q_c))) (Frank-Kamenetskii form of Sec. 8, E = ln(viscosity contrast));
 * T(q_c) = mean of the wedge's six nodal temperatures; r_mid = (r_k + r_k+1)/2. */
typedef struct {
  double E;
  double jump_r;       /* radius of the jump; <= 0 disables it */
  double jump_factor;
} tn_visc_law;

/* Per-wedge viscosity of all levels from nodal temperature T_node_dev (node layout of
 * level 0, doubles).  Stream-ordered. */
tn_status tn_set_temperature(tn_mesh* mesh, const double* T_node_dev, const tn_visc_law* law, void* stream);

/* Copy the current level-h viscosity (wedge layout, doubles) to eta_dev.  Stream-ordered. */
tn_status tn_get_viscosity(const tn_mesh* mesh, int level, double* eta_dev, void* stream);

/* y = (P A P + (I - P)) u on level h (Eq. matfree with Eq. elemmat; the one-point rule, or the
 * mesh's tn_mesh_opts.hg_kappa / radial_quad_points variant of Sec. 4).
 * u_dev[3], y_dev[3]: node layout of level h, type double (TN_F64) or float (TN_F32);
 * y must not alias u.  Stream-ordered.  On levels with N >= 32 the applies use the level's
 * preallocated tile-line buffer (FP64 and FP32), so applies on one mesh must not overlap on the
 * GPU: issue them on one stream, or order their streams with events.  FP32 inputs that start on a
 * 16-byte boundary take the paired-cell kernel, others the square tiles (same result to FP32
 * rounding). */
tn_status tn_apply_A(tn_mesh* mesh, int level, tn_prec prec, const void* const* u_dev, void* const* y_dev,
                     void* stream);

/* q = B P u: divergence onto the pressure space of level h (node layout of level h+1).
 * B[k, (j,d)] = -sum_e V_e psi_k(q_c^e) dN_j/dx_d(q_c^e), psi_k the pressure basis
 * (nested iso-interpolation of the coarse W1 function, Sec. 3); on level 0 with a reference state
 * (tn_set_reference_state) the TALA divergence B_rho P u.  Stream-ordered. */
tn_status tn_apply_B(tn_mesh* mesh, int level, tn_prec prec, const void* const* u_dev, void* q_dev, void* stream);

/* q = B P u exactly as tn_apply_B (same kernels, same result), with the one intermediate that
 * tn_apply_B keeps in mesh-owned scratch -- the fine-level divergence field between the element
 * kernel and the restriction -- in a static device array compiled into the library instead (8 MiB,
 * held by every GPU that loads the library until the process exits).  For callers that cannot
 * allocate device memory at the point of the call, e.g. code running under an allocator that
 * forbids cudaMalloc after start-up; this call makes no cudaMalloc, cudaFree or other allocating
 * call.  FP64 levels with N >= 32 still use the ring buffer that tn_mesh_create preallocated for
 * the tile-line partial sums of the halo-free tiles (no allocation, but mesh-owned memory).
 * The paper has no counterpart; it is an addition of this library.
 * Limit: level h's node layout times the element size (8 B for TN_F64, 4 B for TN_F32) must
 * fit in 8 MiB, else TN_EINVAL with the sizes in tn_last_error().  The mesh's device must be
 * current.  The first call on a device looks up the array's device address (once per device);
 * make that first call before any stream capture.  All calls share the array: calls that
 * overlap on the GPU (other streams, other threads, other meshes) race on it, and calls on one
 * mesh that overlap also race on that mesh's ring buffer.  Nothing in the array needs to start
 * at zero (each call writes every entry it reads).  Stream-ordered. */
tn_status tn_apply_B_static(tn_mesh* mesh, int level, tn_prec prec, const void* const* u_dev, void* q_dev,
                            void* stream);


/* y = P B^T p: gradient of a pressure field (node layout of level h+1) onto the velocity
 * space of level h.  Stream-ordered. */
tn_status tn_apply_BT(tn_mesh* mesh, int level, tn_prec prec, const void* p_dev, void* const* y_dev, void* stream);

/* d = diag(P A P + (I - P)) on level h (3 arrays, node layout), for the mesh's A (one-point rule,
 * hourglass control or the second radial point).  Stream-ordered. */
tn_status tn_diag_A(tn_mesh* mesh, int level, tn_prec prec, void* const* d_dev, void* stream);

/* m = diag(M_{1/eta}) of Eq. (pmass) on the pressure space of level h (node layout of
 * level h+1): sum_e V_e / eta_e psi_k(q_c^e)^2 over the fine wedges.  Stream-ordered. */
tn_status tn_diag_pmass(tn_mesh* mesh, int level, tn_prec prec, void* m_dev, void* stream);

/* n_steps operator steps on level 0 from and to HOST memory.  Step i copies its inputs
 * u_host[3 i + c] (c = 0..2, node layout of level 0) and p_host[i] (node layout of level 1) to
 * the device, computes exactly what tn_apply_A, tn_apply_B, tn_apply_BT and tn_diag_A compute
 * (same kernels, bitwise the same results):
 *   y_A = A u, q = B u, y_BT = B^T p, d = diag(A),
 * and copies them back to out_host[10 i + k]: k = 0..2 y_A, 3 q (level-1 layout), 4..6 y_BT,
 * 7..9 d.  Element type double (TN_F64) or float (TN_F32) throughout.
 * The steps are pipelined over two device buffer sets and two copy streams of the library's own:
 * the copies of one step overlap the compute of its neighbours, which runs on `stream`.  The
 * device buffers (14 vectors per set) are allocated on the first call and kept with the mesh
 * (reallocated when prec changes; freed by tn_mesh_destroy) and zeroed when allocated, so the
 * layout's padding entries (j > N), which no kernel writes, come back as 0.  Host buffers should be pinned
 * (page-locked): with pageable memory the copies do not overlap.  The ten output buffers of one
 * step must not overlap each other, and no output buffer may overlap an input buffer of the call;
 * outputs of different steps may share buffers (all copy-outs run on one library stream in step
 * order, so a later step's result overwrites an earlier one's).  Stream-ordered: the outputs are complete once `stream`
 * reaches the point after this call; the host pointers must stay valid until then.
 * Errors: TN_EINVAL (NULL pointer, n_steps < 0, precision, mesh without a pressure level),
 * TN_ESTATE (viscosity not set), TN_ENOMEM (device buffers), TN_ECUDA. */
tn_status tn_operator_steps_host(tn_mesh* mesh, tn_prec prec, int n_steps, const void* const* u_host,
                                 const void* const* p_host, void* const* out_host, void* stream);

/* Nested iso-interpolation between level h+1 (coarse) and level h (fine), ncomp = 1 or 3
 * arrays: prolongation fine = P coarse, restriction coarse = P^T fine.  With
 * apply_bc != 0 the velocity boundary projector of the target level is applied to
 * the result (multigrid transfers of the constrained space).  Stream-ordered. */
tn_status tn_prolong(tn_mesh* mesh, int level, tn_prec prec, int ncomp, int apply_bc,
                     const void* const* coarse_dev, void* const* fine_dev, void* stream);
tn_status tn_restrict(tn_mesh* mesh, int level, tn_prec prec, int ncomp, int apply_bc,
                      const void* const* fine_dev, void* const* coarse_dev, void* stream);

/* Boussinesq buoyancy right-hand side f = P sum_e V_e Ra T(q_c) r_hat(q_c) N_j(q_c) on level 0
 * (Eq. stokes with the full temperature); f_dev[3] doubles.  With a reference state set
 * (tn_set_reference_state) each wedge's term is weighted by rho(q_c) alpha(q_c), the TALA load
 * Ra rho alpha T' r_hat of Eq. stokes, and T_node_dev is then the perturbation T' of Eq. tsplit.
 * Stream-ordered. */
tn_status tn_buoyancy(tn_mesh* mesh, const double* T_node_dev, double Ra, double* const* f_dev, void* stream);

/* TALA reference state (Sec. 1, Eq. stokes and Eq. mass): the reference density rho_host[k] > 0 and
 * thermal expansivity alpha_host[k] at the level-0 node radii r_k, k = 0 .. N_r - 1 (host arrays,
 * copied; alpha_host NULL = 1; rho_host NULL removes the reference state: the Boussinesq system).
 * With it the mass constraint is div(rho u) = 0, discretised by the product rule at the quadrature
 * point: B_rho[k, (j,d)] = -sum_e V_e psi_k(q_c) (rho(q_c) dN_j/dx_d + rho'(q_c) r_hat_d(q_c) / 6),
 * rho(q_c) = (rho_k + rho_k+1) / 2, rho' = (rho_k+1 - rho_k) / (r_k+1 - r_k), r_hat(q_c) the unit
 * radial direction of the wedge centre; rigid rotations stay an exact null space.  tn_apply_B,
 * tn_apply_B_static, tn_operator_steps_host and tn_stokes_solve use this B, so the saddle matrix
 * [[P A P + I - P, P B^T], [B_rho P, 0]] is not symmetric (FGMRES needs no symmetry);
 * tn_apply_BT, the momentum block and the preconditioner are unchanged, and tn_buoyancy weights
 * its load by rho(q_c) alpha(q_c) (each the mean of the wedge's six nodal values).  Resets the
 * multigrid set-up.  Synchronous.  Errors: TN_EINVAL (NULL mesh, rho <= 0 or non-finite),
 * TN_ENOMEM, TN_ECUDA. */
tn_status tn_set_reference_state(tn_mesh* mesh, const double* rho_host, const double* alpha_host);


/* Measured fused multiply-add throughput of the current device in TFLOP/s (FMA = 2 flops), for
 * prec TN_F64 (DFMA) or TN_F32 (FFMA): independent FMA chains on every SM, timed with CUDA events
 * on `stream`, best of three launches after a warm-up.  The roofline denominator of the element
 * kernels that the FP64 / FP32 pipes bound.  Not a paper operation (a measurement utility).
 * Synchronous; allocates and frees a small device buffer.  Errors: TN_EINVAL, TN_ECUDA. */
tn_status tn_probe_fma_peak(tn_prec prec, double* tflops, void* stream);

/* ------------------------------------------------------------------------------------------
 * Geometric multigrid (Sec. 7): V-cycle over the mesh hierarchy, two pre- and two
 * post-smoothing steps of a degree-2 Chebyshev polynomial in D^-1 K per level (D = the 3x3
 * node-block diagonal of the constrained operator K = P A P + I - P, i.e. block Jacobi),
 * coarsest level solved by conjugate gradients preconditioned with the same D.
 *
 * Chebyshev step (Chebyshev acceleration, Saad, Iterative Methods for Sparse Linear Systems,
 * Alg. 12.1, two iterations) on the interval [cheb_lo, cheb_hi] x lambda, lambda the estimate
 * of the largest eigenvalue of D^-1 K from power_iters power iterations
 * (v <- D^-1 K v / ||D^-1 K v||, lambda = ||D^-1 K v||, Euclidean over unique nodes).
 * The level-0 start vector is v0_dev (3 arrays) or, if NULL, SplitMix64 draws keyed by
 * (seed, canonical layout index, component); level h+1 starts from the restriction of level h's.
 * Coarsest level: D-preconditioned CG from 0 until (r, D^-1 r) <= coarse_rtol^2 (r0, D^-1 r0)
 * or coarse_max_iters; with free-slip on both surfaces the rigid rotations (an exact null space)
 * are projected out of its right-hand side and solution.
 * Transfers: restriction P^T then the coarse boundary projector; prolongation P then the fine
 * boundary projector (as tn_restrict / tn_prolong with apply_bc = 1).
 * Multigrid levels (semi-coarsening): with q = (r_out - r_in) 2^l / (atan(2) r_mid (N_r - 1)) the
 * ratio of radial to lateral cell size, the next level coarsens laterally only if q >= 2,
 * radially only if q <= 1/2, both directions otherwise (or the one still possible); the
 * hierarchy ends when the preferred direction cannot coarsen.  Levels are numbered 0 (finest)
 * upwards; while they coincide with the mesh's levels the mesh's tables are shared.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
  int pre_smooth, post_smooth; /* Chebyshev steps per level (2, 2) */
  int cheb_degree;             /* must be 2 */
  double cheb_lo, cheb_hi;     /* interval factors (0.1, 1.1) */
  int power_iters;             /* 15 */
  int coarse_max_iters;        /* 50 */
  double coarse_rtol;          /* 1e-3 (0: always run coarse_max_iters) */
  int levels;                  /* levels used (0: whole hierarchy) */
  uint64_t seed;               /* internal power-iteration start vector */
} tn_mg_opts;

tn_status tn_mg_default_opts(tn_mg_opts* opts);

/* Diagonals, eigenvalue estimates and workspaces for precision prec (TN_F64 / TN_F32).
 * Needs the viscosity; synchronises the stream; allocates device workspaces owned by the mesh.
 * tn_set_viscosity / tn_set_temperature invalidate it (the next V-cycle or solve re-runs it). */
tn_status tn_mg_setup(tn_mesh* mesh, tn_prec prec, const tn_mg_opts* opts, const void* const* v0_dev, void* stream);
/* lambda estimate of level h after tn_mg_setup (host). */
tn_status tn_mg_lambda(const tn_mesh* mesh, tn_prec prec, int level, double* lambda);
/* z = V(r): one V-cycle from zero on level 0 (3 arrays each, node layout of level 0, type by
 * prec).  Runs tn_mg_setup with the last options if needed.  Stream-ordered, no host sync. */
tn_status tn_vcycle(tn_mesh* mesh, tn_prec prec, const void* const* r_dev, void* const* z_dev, void* stream);

/* ------------------------------------------------------------------------------------------
 * Stokes solve (Sec. 7): FGMRES(restart) (Saad 1993) with right preconditioning by the block
 * upper-triangular P^-1 = [[A^-1, -A^-1 B^T S^-1], [0, S^-1]] of Eq. (block-precond),
 * S^-1 = -diag(M_1/eta)^-1 (Eq. pmass), A^-1 = one V-cycle; classical Gram-Schmidt with one
 * re-orthogonalisation; inner products Euclidean over unique nodes (velocity components and
 * pressure).  The rigid rotations are projected out of the returned velocity when both
 * surfaces are free-slip; the pressure mean is not projected (under free-slip the constant
 * pressure is not an exact null vector of the discrete system).
 * Mode TN_SOLVE_MIXED: FP64 iterative refinement x += ||r|| d with r = b - K x in FP64 and d
 * from an FP32 FGMRES / FP32 V-cycle solve of K d = r / ||r|| to inner_rtol.  Holds the Krylov
 * basis in FP32 (the low-memory mode for the largest shells).
 * Mode TN_SOLVE_F64_PREC32: FP64 FGMRES (FP64 operator, Krylov basis and orthogonalisation)
 * whose preconditioner P^-1 runs in FP32 on the normalised Krylov vector (FP32 Schur step,
 * B^T and V-cycle); FGMRES admits the inexact preconditioner.
 * u, p are outputs (zero initial guess); g may be NULL (zero).  Synchronous.
 * Returns TN_ENOTCONVERGED if ||b - K x|| / ||b|| > rtol on return, or is not a number (stats still
 * filled, converged = 0).  Breakdown exits, each TN_ENOTCONVERGED with the reason in tn_last_error():
 * a non-finite right-hand side returns before the first iteration; a non-finite restart residual or
 * Hessenberg entry (NaN / Inf in the viscosity, the operator or the data) stops FGMRES at that
 * iteration, keeping only the finite part of the update; five restarts in a row that bring the
 * residual less than 0.1 % below its best value so far stop it as stagnation.
 * ---------------------------------------------------------------------------------------- */
typedef enum { TN_SOLVE_F64 = 0, TN_SOLVE_MIXED = 1, TN_SOLVE_F64_PREC32 = 2 } tn_solve_mode;
typedef struct {
  double rtol;          /* 1e-8 relative residual */
  int restart;          /* 30 (1..30) */
  int max_iters;        /* total FGMRES iterations (2000) */
  int mode;             /* tn_solve_mode */
  double inner_rtol;    /* mixed: inner relative tolerance (1e-3) */
  int inner_max_iters;  /* mixed: iterations per inner solve (100) */
  int max_refinements;  /* mixed: outer steps (30) */
} tn_solve_opts;
typedef struct {
  int iterations;       /* FGMRES iterations (summed over inner solves in mixed mode) */
  int refinements;      /* mixed mode outer steps */
  double rel_residual;  /* ||b - K x|| / ||b||, recomputed in FP64 at the end */
  double seconds;       /* host wall time of the call */
  int converged;
} tn_solve_stats;

tn_status tn_solve_default_opts(tn_solve_opts* opts);
tn_status tn_stokes_solve(tn_mesh* mesh, const tn_solve_opts* opts, const double* const* f_dev, const double* g_dev,
                          double* const* u_dev, double* p_dev, tn_solve_stats* stats, void* stream);

/* n independent Stokes solves (1 <= n <= 64, n distinct meshes) advanced in lockstep on one stream:
 * each round enqueues, for every unconverged system, its restart residual or one FGMRES iteration;
 * the V-cycles of all iterating systems run from ONE CUDA graph launch (each system's captured
 * V-cycle a child graph; they run concurrently), then one host synchronisation serves every system.
 * A system leaves the rounds when it converges, breaks down, stalls or is cancelled (its mask bit
 * clears; one combined graph is instantiated per subset of systems that iterate together).  Per
 * system the kernels, their order and the host arithmetic are those of tn_stokes_solve, so each
 * result is bitwise the same as solved alone.  f_dev[i][3], g_dev[i] (g_dev or g_dev[i] may be
 * NULL), u_dev[i][3], p_dev[i], stats[i] (may be NULL) and status[i] (the system's tn_stokes_solve
 * status) per system.  Modes TN_SOLVE_F64 and TN_SOLVE_F64_PREC32 (TN_SOLVE_MIXED: TN_EINVAL).
 * Synchronous.  Returns TN_OK or the first non-OK system status. */
tn_status tn_stokes_solve_batch(tn_mesh* const* meshes, int n, const tn_solve_opts* opts,
                                const double* const* const* f_dev, const double* const* g_dev,
                                double* const* const* u_dev, double* const* p_dev, tn_solve_stats* stats,
                                tn_status* status, void* stream);

/* ------------------------------------------------------------------------------------------
 * Energy equation (Eq. energy) in the nondimensional Boussinesq form of the spherical benchmark
 * runs (Sec. 8): dT/dt + u . grad T = lap T, on level 0, FP64, node layout.  Space: W1 wedges with
 * the one-point rule (Sec. 4), lumped mass m_j = sum_e V_e / 6 and the residual
 *   R_j = sum_e V_e [grad N_j . grad T + N_j(q_c) ubar . grad T + tau_e (ubar . grad N_j)(ubar . grad T)]
 * (diffusion, Galerkin advection, and with supg the streamline-upwind term of SUPG, Brooks and
 * Hughes 1982), all at q_c, ubar the mean of the six nodal velocities, tau_e = h / (2 |ubar|)
 * (coth Pe - 1 / Pe), Pe = |ubar| h / 2, h = (2 V_e)^(1/3).  Time: Heun's method,
 * T* = T - dt M^-1 R(T), T_new = (T + T* - dt M^-1 R(T*)) / 2, on the interior node layers; the two
 * surface layers keep their values (prescribed temperatures).  The paper's own schemes (SUPG,
 * entropy viscosity, MMOC, Sec. 6) are named there without their discrete forms; this is the
 * library's explicit SUPG reading.  The first energy call on a mesh allocates its workspace
 * (five layout vectors), kept until tn_mesh_destroy.
 * ---------------------------------------------------------------------------------------- */
/* R = (K + C(u) + S(u)) T (u_dev NULL: the diffusion K T only; supg 0 drops S).  T_dev, R_dev: node
 * layout of level 0, equal values on node copies; R must not alias T.  Stream-ordered. */
tn_status tn_energy_residual(tn_mesh* mesh, const double* T_dev, const double* const* u_dev, int supg, double* R_dev,
                             void* stream);
/* n_steps Heun steps of size dt with the fixed velocity u_dev (NULL: diffusion only), T_dev updated
 * in place.  Stable for dt <= tn_energy_stable_dt and an advective Courant number below ~1.
 * Stream-ordered (the first call synchronises once to set up the workspace). */
tn_status tn_energy_steps(tn_mesh* mesh, double* T_dev, const double* const* u_dev, double dt, int n_steps, int supg,
                          void* stream);
/* Diagnostics (synchronous; either output may be NULL): nu_top = the consistent diffusive heat flux
 * through the outer surface (the residual K T summed over its nodes) divided by the same for the
 * conductive profile T_c = r_in (r - r_out) / (r (r_in - r_out)); v_rms = sqrt(sum_j m_j |u_j|^2 /
 * sum_j m_j) over the unique nodes. */
tn_status tn_energy_diagnostics(tn_mesh* mesh, const double* T_dev, const double* const* u_dev, double* nu_top,
                                double* v_rms, void* stream);
/* Largest stable diffusion substep: 1.5 / (1.1 lambda), lambda the largest eigenvalue of M^-1 K on
 * the interior layers from 30 power iterations (cached per mesh).  Synchronous. */
tn_status tn_energy_stable_dt(tn_mesh* mesh, double* dt, void* stream);

/* Coupled Stokes-energy time loop: n_steps steps of
 *   viscosity exp(E (1/2 - T)) from T (tn_set_temperature), Boussinesq load Ra T r_hat (tn_buoyancy),
 *   Stokes solve to rtol in the given mode (tn_stokes_solve) -> u, p,
 *   diagnostics of (T, u) (tn_energy_diagnostics), then the energy update over
 *   dt = cfl h_min / max |u| (h_min the smallest radial or lateral node spacing) in
 *   ceil(dt / stable substep) Heun substeps; opts.dt > 0 / opts.substeps > 0 fix them instead.
 * T_dev (in / out) must hold the surface temperatures; u_dev, p_dev receive the last solve.
 * stats (may be NULL) gets one entry per step.  Synchronous.  Errors of the solve are returned
 * (TN_ENOTCONVERGED stops the loop after that step's solve). */
typedef struct {
  double Ra;         /* Rayleigh number (1e5) */
  double E;          /* ln(viscosity contrast) of exp(E (1/2 - T)) (ln 100) */
  double cfl;        /* advective Courant number of a step (0.5) */
  int supg;          /* streamline-upwind term (1) */
  int mode;          /* tn_solve_mode of the Stokes solves (TN_SOLVE_MIXED) */
  double rtol;       /* Stokes relative residual (1e-8) */
  double dt;         /* > 0: fixed step instead of the CFL step (0) */
  int substeps;      /* > 0: fixed Heun substeps per step instead of the stability bound (0) */
} tn_convection_opts;
typedef struct {
  double time, dt;          /* model time after the step, step size */
  int substeps;             /* Heun substeps of the energy update */
  int stokes_iterations;
  double rel_residual;      /* of the Stokes solve */
  double nu_top, v_rms, u_max;   /* diagnostics of the step's (T, u) before the update */
  double stokes_seconds, energy_seconds;  /* host wall time of the two halves */
} tn_convection_step_stats;
tn_status tn_convection_default_opts(tn_convection_opts* opts);
tn_status tn_convection_steps(tn_mesh* mesh, double* T_dev, double* const* u_dev, double* p_dev, int n_steps,
                              const tn_convection_opts* opts, tn_convection_step_stats* stats, void* stream);

/* ------------------------------------------------------------------------------------------
 * Serving: continuous batching of Stokes solves (the paper has no serving layer).
 * tn_server_submit queues a request and returns at once.  max_active worker threads, each
 * with its own stream, take the first queued request that fits the device-memory budget
 * (memory_fraction x free memory when the server was created) and run tn_stokes_solve on it,
 * so solves of different requests overlap on the GPU.  Mesh hierarchies stay resident per
 * shape and are reused; idle ones are evicted least recently used when a new shape needs
 * room.  A request larger than the whole budget completes at once with status TN_ENOMEM.
 * Each request's result is independent of the other requests running (own mesh, vectors and
 * stream, fixed-order reductions).
 * Request temperature: T = r_in (r - r_out) / (r (r_in - r_out))
 *   + t_amplitude cos(t_order phi) P_l^m(cos theta) / max|P_l^m| sin(pi (r - r_in) / (r_out - r_in)),
 * l = t_degree, m = t_order; viscosity exp(E (1/2 - T)); buoyancy Ra T r_hat; free-slip.
 * ---------------------------------------------------------------------------------------- */
typedef struct tn_server tn_server;
typedef struct {
  int max_active;          /* concurrent solves (4) */
  double memory_fraction;  /* share of the free device memory the server may hold (0.8) */
  int mode;                /* tn_solve_mode of every solve (TN_SOLVE_MIXED) */
  double rtol;             /* 1e-8 */
  int keep_solutions;      /* 1: keep a host copy of every solution for tn_server_solution (0) */
  int eta_storage;         /* tn_mesh_opts.eta_storage of every request's mesh (TN_ETA_F32) */
  double hg_kappa;         /* tn_mesh_opts.hg_kappa of every request's mesh (0: the plain one-point A) */
  int radial_quad_points;  /* tn_mesh_opts.radial_quad_points of every request's mesh (1) */
  int max_batch;           /* 1..64 (1): a worker that takes a request also takes up to max_batch - 1
                            * queued requests of the same shape (as far as the memory budget admits)
                            * and solves them in lockstep with tn_stokes_solve_batch (modes TN_SOLVE_F64
                            * and TN_SOLVE_F64_PREC32; TN_SOLVE_MIXED solves them one after another) */
} tn_server_opts;
typedef struct {
  int lateral_level, radial_layers;
  double r_in, r_out;
  double E;                /* ln(viscosity contrast) */
  double Ra;
  int t_degree, t_order;
  double t_amplitude;
} tn_request;
typedef struct {
  int state;               /* 0 queued, 1 running, 2 done */
  int status;              /* result of the solve once done (TN_OK, TN_ENOTCONVERGED, TN_ENOMEM, ...) */
  int iterations, refinements;
  double rel_residual;
  double t_submit, t_start, t_end;  /* seconds since tn_server_create (host clock) */
  int batch;               /* systems in the lockstep batch that solved it (0: solved alone) */
} tn_result;

tn_status tn_server_default_opts(tn_server_opts* opts);
/* Starts the worker threads on the current device.  opts may be NULL. */
tn_status tn_server_create(const tn_server_opts* opts, tn_server** out);
tn_status tn_server_submit(tn_server* srv, const tn_request* req, uint64_t* ticket);
/* TN_OK and the result if the request is done, TN_EBUSY (result holds its state) otherwise. */
tn_status tn_server_poll(tn_server* srv, uint64_t ticket, tn_result* res);
/* Blocks until the request is done. */
tn_status tn_server_wait(tn_server* srv, uint64_t ticket, tn_result* res);
/* Host copy of a finished solution (keep_solutions = 1): u_host 3 x n_layout of level 0
 * (component-major), p_host n_layout of level 1, layouts as for a mesh of the request's shape. */
tn_status tn_server_solution(tn_server* srv, uint64_t ticket, double* u_host, double* p_host);
tn_status tn_server_stats(tn_server* srv, int* queued, int* running, int* resident, double* reserved_bytes);
/* Cancel a request: a queued one completes at once with status TN_ECANCELED and never runs; a
 * running one stops at its next Krylov iteration (the solver polls the flag once per iteration),
 * completes with TN_ECANCELED and frees its slot and vectors; a finished one is left as it is.
 * Returns TN_OK, or TN_EINVAL for an unknown ticket.  Thread-safe. */
tn_status tn_server_cancel(tn_server* srv, uint64_t ticket);
/* Finishes every queued request, then stops the workers and frees everything. */
tn_status tn_server_destroy(tn_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* TERRA_WEDGE_H */
