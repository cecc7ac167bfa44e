/*
 * hx — matrix-free high-order Helmholtz / Poisson operator and Jacobi-PCG on
 * one NVIDIA B300 (sm_103a).  C ABI of libhx.so.
 *
 * The operator is A = alpha M + K(nu) on a continuous Q_p space over a mesh of
 * trilinear hexahedra, with the nodal Gauss-Lobatto-Legendre basis and tensor
 * Gauss quadrature with q points per direction:
 *   M_ij = int phi_i phi_j dx                      (Sec. 2, Eq. (vectorMass))
 *   K_ij = int nu grad phi_i . grad phi_j dx       (Sec. 2, Eq. (vectorDiffusion);
 *                                                   element form Sec. 3.1, Eqs. (localStiffness)-(localStiffnessQuadrature))
 * i.e. the system A u = b with A = c M + L, c >= 0, of Sec. 5.2, applied
 * matrix-free by sum factorization (Sec. 3.1) and solved with conjugate
 * gradients (Sec. 5, Sec. 5.3) preconditioned by the diagonal of A.
 *
 * Conventions (readings where the paper is silent):
 *   - reference cube [-1,1]^3; local node and quadrature-point order is
 *     lexicographic with the first reference coordinate fastest;
 *   - J_ij = dx_i/dxi_j, stiffness coefficient nu w detJ J^-1 J^-T;
 *   - Dirichlet DoFs are eliminated symmetrically: the constrained operator is
 *     A_c = P A P + (I - P), P zeroing Dirichlet DoFs; solves use b_c = P b;
 *   - element corners are ordered c = cx + 2 cy + 4 cz (corner c at reference
 *     point (2cx-1, 2cy-1, 2cz-1)).
 *
 * Memory and streams: arguments documented "device" are pointers into the
 * current CUDA device's global memory, owned by the caller and left
 * untouched by the library except where written as outputs.  "host" pointers
 * are ordinary CPU memory (pinned memory gives faster copies).  The library
 * allocates and owns its own workspaces (restriction maps, geometric factors,
 * E-vectors, CG vectors) in *_create (CG vectors at the first solve) and frees
 * them in *_destroy.  Calls taking a `stream` (a cudaStream_t passed as void*,
 * NULL = legacy default stream) enqueue their work on it and return without
 * waiting, except where noted.
 *
 * Errors: every call returns an hx_status; 0 is success.  On failure the
 * thread-local message hx_last_error() says what went wrong.  No call aborts,
 * throws or exits.  Supported orders: 1 <= p <= 8 with q = p+1 or q = p+2.
 */
#ifndef HX_H
#define HX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HX_API __attribute__((visibility("default")))
#else
#define HX_API
#endif

typedef int hx_status;

#define HX_OK 0
#define HX_ERR_ARG (-1)            /* invalid argument (null pointer, bad size, out-of-range index) */
#define HX_ERR_CUDA (-2)           /* a CUDA runtime call failed */
#define HX_ERR_OOM (-3)            /* device memory allocation failed */
#define HX_ERR_INVALID_MESH (-4)   /* detJ <= 0 at some quadrature point */
#define HX_ERR_NOT_CONVERGED (-5)  /* CG hit max_it before the tolerance */
#define HX_ERR_BREAKDOWN (-6)      /* CG breakdown: p^T A p <= 0 or a non-finite value */
#define HX_ERR_UNSUPPORTED (-7)    /* (p, q) or a size outside what is built */

#define HX_GEOM_STORED 0   /* factors m, G stored at every quadrature point (Sec. 3.1: J stored at points) */
#define HX_GEOM_ONTHEFLY 1 /* factors recomputed from the 8 element vertices at every apply */

typedef struct hx_mesh hx_mesh;
typedef struct hx_op hx_op;

/* Result of a solve (all fields filled whatever the return status). */
typedef struct hx_solve_info {
  int iterations;            /* CG iterations performed */
  int status;                /* HX_OK, HX_ERR_NOT_CONVERGED or HX_ERR_BREAKDOWN */
  double rel_residual;       /* ||r_k||_2 / ||P b||_2 of the CG recurrence residual */
  double true_rel_residual;  /* ||P b - A_c x||_2 / ||P b||_2, recomputed with one extra apply */
  double b_norm;             /* ||P b||_2 */
  int kernel_launches;       /* kernels this solve enqueued (CUDA-graph replays included) */
  int refinements;           /* hx_solve_pcg_mixed: FP64 refinement steps (0 for the FP64 solves) */
} hx_solve_info;

/* Library version (major * 10000 + minor * 100 + patch). */
HX_API int hx_version(void);

/* Message of the last failed call on this thread ("" if none).  Valid until the next call. */
HX_API const char* hx_last_error(void);

/*
 * Mesh of trilinear hexahedra carrying a Q_p space (Sec. 3: mapped hexahedra,
 * nodal Gauss-Lobatto tensor-product basis; Sec. 3.1: the element restriction
 * over which the element-by-element sum of the operator action runs).
 *   p, q          order and Gauss points per direction (1 <= p <= 8, q in {p+1, p+2})
 *   n_vert        number of vertices; vert_xyz: host, n_vert x 3 doubles (x, y, z per vertex)
 *   n_elem        number of elements; elem_vert: host, n_elem x 8 vertex ids (corner order above)
 *   n_dof         number of global DoFs (L-vector length)
 *   restriction   host, n_elem x (p+1)^3 global DoF ids in [0, n_dof), local node order
 *                 lexicographic; the caller guarantees it is conforming (shared nodes share ids)
 *   dirichlet     host, n_dof bytes, nonzero = Dirichlet (eliminated) DoF; NULL = none
 *   out           receives the new mesh (NULL on failure)
 * Copies everything to the device; the host arrays can be freed on return.
 * Errors: HX_ERR_ARG (null/invalid sizes, ids out of range, a DoF in no element),
 * HX_ERR_UNSUPPORTED (p, q, or n_elem (p+1)^3 >= 2^31), HX_ERR_OOM, HX_ERR_CUDA.
 * Synchronous.
 */
HX_API hx_status hx_mesh_create(int p, int q, int64_t n_vert, const double* vert_xyz, int64_t n_elem,
                                const int64_t* elem_vert, int64_t n_dof, const int64_t* restriction,
                                const uint8_t* dirichlet, hx_mesh** out);

/*
 * Structured nx x ny x nz mesh (elements and vertices lexicographic, x fastest)
 * with the vertex positions given: vert_xyz is host, (nx+1)(ny+1)(nz+1) x 3.
 * The library numbers the global DoFs lexicographically over the
 * (p nx + 1) x (p ny + 1) x (p nz + 1) node grid (x fastest) and marks every
 * DoF on the boundary of the index box as Dirichlet.  Errors as hx_mesh_create.
 */
HX_API hx_status hx_mesh_create_structured(int nx, int ny, int nz, int p, int q, const double* vert_xyz,
                                           hx_mesh** out);

/*
 * As hx_mesh_create_structured, with the Dirichlet DoFs on a chosen set of box
 * faces: bit 0 x = min, bit 1 x = max, bit 2 y = min, bit 3 y = max, bit 4 z = min,
 * bit 5 z = max (63 = all faces; 0 = pure Neumann).  An operator with alpha = 0 on a
 * mesh without Dirichlet DoFs is the pure-Neumann Poisson operator of the pressure
 * step (Sec. 4.2): its solves remove the mean of b, orthogonalize every
 * preconditioned residual against the constants (Sec. 5.3) and return the
 * solution with zero mean, int x dx = 0 (Eq. (meanZero)).
 */
HX_API hx_status hx_mesh_create_box(int nx, int ny, int nz, int p, int q, const double* vert_xyz,
                                    int dirichlet_faces, hx_mesh** out);

/* Frees the mesh (NULL is ignored).  Operators built on it must be destroyed first. */
HX_API void hx_mesh_destroy(hx_mesh* mesh);

/* Sizes of a mesh; any output pointer may be NULL. */
HX_API hx_status hx_mesh_info(const hx_mesh* mesh, int64_t* n_elem, int64_t* n_dof, int* p, int* q);

/*
 * Physical coordinates of the quadrature points (the points xi of Sec. 3.1
 * mapped by the trilinear element map).  xyz: device, n_elem x q^3 x 3
 * doubles, point order lexicographic.  Stream-ordered.
 */
HX_API hx_status hx_mesh_qpoint_coords(const hx_mesh* mesh, double* xyz, void* stream);

/* Physical coordinates of every global DoF (GLL node).  xyz: device, n_dof x 3.  Stream-ordered. */
HX_API hx_status hx_mesh_node_coords(const hx_mesh* mesh, double* xyz, void* stream);

/*
 * Operator A = alpha M + K(nu) (Sec. 5.2, A = c M + L) on `mesh`.
 *   alpha      mass coefficient (>= 0 for an SPD/SPSD operator; e.g. 1/dt, 0 for Poisson)
 *   nu         constant viscosity, used when nu_q is NULL
 *   nu_q       device, n_elem x q^3 per-quadrature-point viscosity, or NULL; copied
 *   geom_mode  HX_GEOM_STORED: precompute m = alpha w detJ and G = nu w detJ J^-1 J^-T
 *              at every point ([E][7][q^3] doubles, Sec. 3.1 stored-J variant);
 *              HX_GEOM_ONTHEFLY: recompute them from the element vertices at each apply
 *   stream     stream for the setup kernels (geometric factors)
 * The diagonal of A (for Jacobi) is assembled by the first call that needs it
 * (a solve, hx_op_diagonal).  Returns HX_ERR_INVALID_MESH
 * when detJ <= 0 at some quadrature point.  Synchronizes `stream` before returning.
 */
HX_API hx_status hx_op_create(hx_mesh* mesh, double alpha, double nu, const double* nu_q, int geom_mode,
                              void* stream, hx_op** out);

/*
 * Replace the coefficients of an existing operator: updates the stored
 * factors m = alpha w detJ, G = nu w detJ J^-1 J^-T (Sec. 3.1); the diagonal
 * follows at the next call that needs it.  Use: the time step 1/alpha or the
 * viscosity changes between the Helmholtz solves of successive time steps
 * (Sec. 4.2, Sec. 5.3).  Same meaning of alpha, nu, nu_q as hx_op_create; an
 * HX_GEOM_ONTHEFLY operator takes a nu_q field only if it was created with one.
 * With stored factors and constant coefficients, both nonzero before and after,
 * the factors are scaled in place by alpha'/alpha and nu'/nu (m is linear in
 * alpha, G in nu; one rounding per update) and the diagonal is combined from
 * its mass and stiffness parts; a zero coefficient, a nu field, or 64 such
 * updates in a row recompute the factors from the geometry.  Allocates
 * nothing; stream-ordered.
 */
HX_API hx_status hx_op_set_coefficients(hx_op* op, double alpha, double nu, const double* nu_q, void* stream);

/* Number of kernels the operator has enqueued since creation (graph replays counted per kernel). */
HX_API int64_t hx_op_launch_count(const hx_op* op);

/* Sizes of the mesh an operator is built on; any output pointer may be NULL. */
HX_API hx_status hx_op_info(const hx_op* op, int64_t* n_elem, int64_t* n_dof, int* p, int* q);

/* Frees the operator (NULL is ignored).  Touches only the operator's own memory, so it is
 * safe after its mesh has been destroyed (the operator can no longer be used then). */
HX_API void hx_op_destroy(hx_op* op);

/*
 * y = A x (constrained = 0) or y = A_c x = P A P x + (I - P) x (constrained = 1),
 * matrix-free: gather through the element restriction, sum-factorized
 * contractions with B and D (Sec. 3.1, Eqs. (B1D), (D1D), (sumFactorized),
 * (tensorGradient)), pointwise factors, transposed contractions, and an
 * atomic-free element-to-global sum in a fixed order (bitwise reproducible).
 * x, y: device, n_dof doubles each; must not overlap.  Stream-ordered.
 */
HX_API hx_status hx_op_apply(hx_op* op, const double* x, double* y, int constrained, void* stream);

/*
 * diag: device, n_dof doubles <- the exact diagonal of A (same quadrature),
 * assembled sum-factorized; with constrained = 1 the Dirichlet entries are 1
 * (the diagonal of A_c).  Stream-ordered.
 */
HX_API hx_status hx_op_diagonal(hx_op* op, double* diag, int constrained, void* stream);

/*
 * Load vector b_i = (f, phi_i) = sum_K sum_q w_q detJ_q f_q phi_i(xi_q), the
 * right-hand side of the weak form (Sec. 3, Eq. (weak-stokes), one scalar
 * component).  f_q: device, n_elem x q^3 values of f at the quadrature points
 * (see hx_mesh_qpoint_coords); b: device, n_dof.  Stream-ordered.
 */
HX_API hx_status hx_op_load_vector(hx_op* op, const double* f_q, double* b, void* stream);

/*
 * Jacobi-preconditioned CG (Sec. 5, Sec. 5.3; Jacobi = diagonal of A_c) for
 * A_c x = P b.  Stops when ||r_k||_2 <= rtol ||P b||_2 (recurrence residual) or
 * after max_it iterations (max_it = 0: no iteration; HX_ERR_NOT_CONVERGED
 * unless the initial residual already meets the tolerance, as when P b = 0).
 *   b         device, n_dof (entries at Dirichlet DoFs are ignored)
 *   x         device, n_dof; input initial guess if use_x0 != 0 (Dirichlet
 *             entries taken as 0), else ignored; output solution (0 at Dirichlet DoFs)
 *   info      host, filled on return (may be NULL)
 * All scalars stay on the device; iterations run in a CUDA graph and the
 * host only polls a status word.  Waits for `stream`'s prior work and
 * returns after the solution is written (synchronous).
 * Returns HX_OK, HX_ERR_NOT_CONVERGED or HX_ERR_BREAKDOWN (x then holds the
 * last iterate), or an argument / CUDA error.
 */
HX_API hx_status hx_solve_pcg(hx_op* op, const double* b, double* x, double rtol, int max_it, int use_x0,
                              void* stream, hx_solve_info* info);

/*
 * As hx_solve_pcg with b and x in host memory: after the caller's prior work
 * on `stream` (e.g. an hx_op_set_coefficients), copies b (and x0) to the
 * device, solves, and copies x back.  b_host, x_host: host, n_dof doubles.
 * Synchronous.
 */
HX_API hx_status hx_solve_pcg_host(hx_op* op, const double* b_host, double* x_host, double rtol, int max_it,
                                   int use_x0, void* stream, hx_solve_info* info);

/*
 * Mixed-precision solve of A_c x = P b to the FP64 relative residual rtol:
 * iterative refinement whose residual r = P b - A_c x, update x += |r| d and
 * solution accumulate in FP64, while each correction d solves A_c d = r / |r|
 * with an FP32 PCG (FP32 operator apply: the same sum-factorized kernels in
 * FP32 with the FP32 rounding of the stored factors, or FP32 on-the-fly
 * geometry) to the relative residual inner_rtol (e.g. 1e-5).  The inner
 * preconditioner follows hx_op_set_preconditioner: Jacobi (the diagonal of the
 * FP32 operator, computed in FP32), the collocated mass, or the LOR multigrid
 * V-cycle run in FP32 on FP32 copies of its levels.
 * Not in the paper; it trades the B300's 1:64 FP64:FP32 rate for a few FP64
 * residual applies.  max_it caps the total inner iterations; the solve also
 * stops with HX_ERR_NOT_CONVERGED when two refinement steps in a row fail to
 * halve the residual.  info->iterations = inner iterations in total,
 * info->refinements = FP64 refinement steps, rel_residual = true_rel_residual =
 * the final FP64 residual.  Arguments and synchronization as hx_solve_pcg.
 * The first call allocates the FP32 workspace (FP32 factors, vectors).
 */
HX_API hx_status hx_solve_pcg_mixed(hx_op* op, const double* b, double* x, double rtol, int max_it,
                                    double inner_rtol, void* stream, hx_solve_info* info);

/*
 * The FP32 operator of the mixed-precision solve, constrained form:
 * y = P A P x + (I - P) x in FP32.  x, y: device, n_dof floats.  Stream-ordered.
 */
HX_API hx_status hx_op_apply_f32(hx_op* op, const float* x, float* y, void* stream);

/*
 * The FP32 element kernel of the mixed-precision solve (the paper has no counterpart; all
 * compute the same FP32 operator as hx_op_apply_f32, to FP32 rounding):
 *   HX_F32_COLLOCATED     interpolate with B, differentiate with the q x q collocation matrix
 *                         Dh at the Gauss points (the FP64 kernel's form), factors staged by
 *                         one bulk copy per block for p <= 4
 *   HX_F32_DIRECT_STAGED  the "B/D-direct" form (u, du/dxi by B and D along each direction,
 *                         intermediates written and read once), element-interleaved shared
 *                         memory, restriction and stored factors brought in by bulk (TMA)
 *                         copies at block start; stored factors only
 *   HX_F32_DIRECT         the same with the factors read from global memory (or recomputed
 *                         from the vertices for on-the-fly geometry)
 *   HX_F32_MMA_BF16       the B/D-direct form with every 1D contraction on the tensor cores
 *                         (warp-level mma.sync m16n8k16, BF16 operands, FP32 accumulation):
 *                         operands rounded to BF16 (8 significant bits), so the operator is
 *                         accurate to ~1e-2 relative, not to FP32; stored factors only
 *   HX_F32_MMA_BF16X3     the same with each operand split into a high and a low BF16 part and
 *                         three products accumulated (hi*hi + hi*lo + lo*hi, ~16 significant
 *                         bits, ~1e-4 relative); stored factors only
 *   HX_F32_AUTO           (default) the fastest of the FP32-accurate candidates -- kernel form
 *                         (HX_F32_COLLOCATED, HX_F32_DIRECT_STAGED, HX_F32_DIRECT) and, for the
 *                         direct forms with stored factors, tile shape (half, the default or
 *                         twice the elements per block, where the block stays within 1024
 *                         threads and the shared memory) -- for this order, quadrature, geometry
 *                         mode and size class (log2 of the element count), timed once per
 *                         process by the operator's first FP32 set-up (one warm-up and three
 *                         timed launches of each candidate, CUDA events) and cached
 * hx_op_set_f32_kernel selects one kind with its default tile (HX_ERR_ARG for an unknown kind,
 * HX_ERR_UNSUPPORTED for a stored-factor kind with on-the-fly geometry); it takes effect at the
 * next FP32 set-up.  hx_op_f32_kernel reports the kernel in use (*kind = -1 before the first
 * FP32 set-up), when block_elems is not NULL its elements per block (-1 for the kinds with a
 * fixed block), and when ms is not NULL the autotuner's average time per launch of each kind's
 * fastest tile in ms (ms[kind] for kinds 0..2, -1 where not timed).  Host-side only.
 */
#define HX_F32_AUTO (-1)
#define HX_F32_COLLOCATED 0
#define HX_F32_DIRECT_STAGED 1
#define HX_F32_DIRECT 2
#define HX_F32_MMA_BF16 3
#define HX_F32_MMA_BF16X3 4
HX_API hx_status hx_op_set_f32_kernel(hx_op* op, int kind);
/*
 * Tile variant of a kind selected with hx_op_set_f32_kernel (test and tuning hook): -1, 0, +1
 * for half, the default and twice the elements per block of HX_F32_DIRECT_STAGED and
 * HX_F32_DIRECT with stored factors; other kinds and HX_F32_AUTO ignore it.  HX_ERR_ARG outside
 * -1..1, HX_ERR_UNSUPPORTED for a nonzero tile with on-the-fly geometry; a variant the order
 * does not have (more than 8 elements or 1024 threads per block) makes the next FP32 set-up
 * return HX_ERR_UNSUPPORTED.  Takes effect at the next FP32 set-up.  Host-side only.
 */
HX_API hx_status hx_op_set_f32_tile(hx_op* op, int tile);
HX_API hx_status hx_op_f32_kernel(const hx_op* op, int* kind, int* block_elems, float* ms /* 3 entries or NULL */);

/*
 * Failure-detection hook (the paper has no counterpart).  For p <= 4 with stored
 * factors the FP32 operator kernel stages each block's factors into shared memory
 * with one bulk (TMA) copy completed on an mbarrier, and waits for it with a bounded
 * number of mbarrier try_wait attempts (default 65536); the HX_F32_DIRECT_STAGED kernel also
 * copies each block's restriction that way and waits for it (same bound) before its gather.  A block whose wait gives up
 * raises the operator's device error flag, skips its remaining stages and stores,
 * and before it exits waits again with a far larger bound, so that no copy is still
 * writing its shared memory.  hx_solve_pcg_mixed reports a raised flag as HX_ERR_CUDA
 * ("... timed out").  attempts (>= 0, else HX_ERR_ARG) sets the first wait's bound
 * for this operator's later mixed solves and FP32 applies; 0 makes every such wait
 * give up at once (the copies themselves complete normally), which tests use to
 * check that the failure surfaces as a status and that the next solve with the
 * default bound runs normally.  Host-side only; drops the captured inner-CG graph.
 */
HX_API hx_status hx_op_set_wait_limit(hx_op* op, int attempts);

/*
 * Preconditioners of the PCG solves (Sec. 5).
 *   HX_PREC_JACOBI           z = diag(A)^-1 r, the exact diagonal of alpha M + nu K (default)
 *   HX_PREC_COLLOCATED_MASS  z = (alpha Mc)^-1 r, Mc the mass matrix integrated with the
 *                            Gauss-Lobatto rule at the nodes of the nodal basis, which is
 *                            diagonal and spectrally equivalent to M independently of h and
 *                            p (Sec. 5.1): the preconditioner of mass-dominated solves
 *   HX_PREC_LOR              z = P_k(D^-1 A_LOR) D^-1 r: `degree` = k steps of the Chebyshev
 *                            iteration for A_LOR z = r with Jacobi scaling D = diag(A_LOR),
 *                            on the interval [b / k^2, b], b the Gershgorin bound of
 *                            D^-1 A_LOR.  A_LOR = alpha M_LOR + nu K_LOR is the low-order
 *                            (Q1, 2 Gauss points per direction) discretization on the mesh
 *                            that cuts every element along its Gauss-Lobatto points, assembled
 *                            and stored as a sparse matrix (Sec. 5.2).  The paper solves
 *                            A_LOR with multigrid and Schwarz methods; here a fixed
 *                            polynomial keeps the preconditioner symmetric and linear for CG.
 *                            Constant nu only.
 *   HX_PREC_LOR_MC           as HX_PREC_LOR with A_LOR = alpha Mc + nu K_LOR: the collocated
 *                            mass of Sec. 5.1 in place of the Q1 mass.  Not in the paper:
 *                            the Q1 mass is a poor match of M when alpha dominates (iteration
 *                            counts double against Jacobi at alpha = 1000, nu = 1e-2), Mc is a
 *                            good one, and the stiffness part is unchanged.
 *   HX_PREC_LOR_MG           z = one symmetric V-cycle for A_LOR z = r, A_LOR = alpha Mc +
 *                            nu K_LOR, on meshes from hx_mesh_create_box/structured (the
 *                            paper's structured geometric multigrid on the LOR matrix,
 *                            Sec. 5.2).  The (pN+1)^3 LOR grid is coarsened vertex-centred
 *                            while every dimension is odd and >= 5; trilinear interpolation P
 *                            of the logical grid, Galerkin coarse operators P^T A P (27-point
 *                            stencils), `degree` Chebyshev-Jacobi smoothing steps on
 *                            [b / 10, b] before and after the coarse correction (the paper
 *                            smooths with ordered ILU), 16 Chebyshev steps on [b / 256, b] on
 *                            the coarsest grid.  HX_ERR_UNSUPPORTED on other meshes.
 * Jacobi and collocated mass use z = r in Dirichlet rows; A_LOR has identity rows there.
 */
#define HX_PREC_JACOBI 0
#define HX_PREC_COLLOCATED_MASS 1
#define HX_PREC_LOR 2
#define HX_PREC_LOR_MC 3
#define HX_PREC_LOR_MG 4

/*
 * alpha Mc as a vector (Sec. 5.1): diag[i] = alpha sum over elements K and local nodes
 * l = (a, b, c) of K with global id i of w_a w_b w_c detJ_K(xi_l), w the Gauss-Lobatto
 * weights.  Unconstrained (Dirichlet rows keep their value).  diag: device, n_dof.
 * Stream-ordered.
 */
HX_API hx_status hx_op_collocated_mass(hx_op* op, double* diag, void* stream);

/*
 * Select the preconditioner of hx_solve_pcg, hx_solve_pcg_host, hx_solve_pcg_mixed and
 * batched solves of this operator (kind: HX_PREC_*; degree: Chebyshev steps of
 * HX_PREC_LOR / HX_PREC_LOR_MC, smoothing steps of HX_PREC_LOR_MG, 1..64, ignored
 * otherwise).  The choice follows later
 * hx_op_set_coefficients calls; a batch keeps the preconditioners its operators had
 * when it was created.
 * Errors: HX_ERR_ARG (unknown kind, degree out of range, HX_PREC_COLLOCATED_MASS with
 * alpha <= 0, also from a later hx_op_set_coefficients with alpha <= 0);
 * HX_ERR_UNSUPPORTED (a LOR form on an operator with a nu field, a LOR row with more
 * than 64 distinct columns, HX_PREC_LOR_MG on a mesh without a logical grid;
 * mixed-precision solves reject HX_PREC_LOR and HX_PREC_LOR_MC).
 * The first selection of a LOR form allocates and builds the sparsity pattern (two
 * synchronizations of `stream`) and, for HX_PREC_LOR_MG, the grid hierarchy; later calls
 * are stream-ordered.  Device memory: HX_PREC_LOR / HX_PREC_LOR_MC hold A_LOR twice, as
 * CSR (12 B per entry, 27 entries per interior row of a structured mesh) and as the
 * sliced-ELL copy the Chebyshev steps read (slices of 32 rows, column-major, padded to
 * the slice's longest row), plus 4 work vectors; HX_PREC_LOR_MG holds 27 stencil values
 * per grid node on every level (the fine level has n_dof nodes, each coarser ~1/8 of the
 * one above) and 6 work vectors per level.  A failed allocation leaves the previous
 * preconditioner selected and may be retried.
 */
HX_API hx_status hx_op_set_preconditioner(hx_op* op, int kind, int degree, void* stream);

/*
 * The assembled low-order refined matrix A_LOR of the operator's alpha, nu (Sec. 5.2; the
 * HX_PREC_LOR_MC form when that preconditioner is selected) in
 * CSR form with the Dirichlet rows and columns eliminated (unit diagonal in Dirichlet
 * rows), columns sorted within each row.  *nnz receives the number of stored entries;
 * row_off (device, n_dof + 1 int64), col (device, nnz int32) and val (device, nnz
 * doubles) receive copies when not NULL (call with NULLs first to size them).
 * Builds the matrix when no HX_PREC_LOR was selected (errors as hx_op_set_preconditioner).
 */
HX_API hx_status hx_op_lor_csr(hx_op* op, int64_t* nnz, int64_t* row_off, int* col, double* val, void* stream);

/*
 * z = the current preconditioner applied to r (as one PCG step applies it).
 * r, z: device, n_dof.  Sets up the solver workspace on first use.  Stream-ordered.
 */
HX_API hx_status hx_op_precond_apply(hx_op* op, const double* r, double* z, void* stream);

/*
 * Adjoint gradient contraction (not in the paper, which solves forward problems):
 * for a loss L(u) of the solution of A_c(nu) u = P b(f), with lam solving
 * A_c lam = P dL/du (hx_solve_pcg with b = dL/du), writes at every quadrature point
 *   dnu_q[e][q] = dL/dnu_q = -w_q detJ_q (J^-T grad lam)_q . (J^-T grad u)_q
 *   df_q[e][q]  = dL/df_q  =  w_q detJ_q lam(x_q)      (f_q as in hx_op_load_vector)
 * by the operator's forward sum-factorized contractions applied to u and lam and a
 * pointwise contraction with the geometric factor recomputed from the vertices.
 * u, lam: device, n_dof (Dirichlet entries read as zero); dnu_q, df_q: device,
 * n_elem x q^3.  Stream-ordered.
 */
HX_API hx_status hx_op_gradient(hx_op* op, const double* u, const double* lam, double* dnu_q, double* df_q,
                                void* stream);

/*
 * Batched solves.  A batch binds n independent problems A_i x_i = b_i (each an
 * operator with its own mesh, order and coefficients: the three velocity
 * Helmholtz solves and the pressure Poisson solve of one projection step,
 * Sec. 4.2 and Sec. 5.3, or unrelated instances) and builds one CUDA graph in
 * which every instance's whole Jacobi-PCG — initialization, the iterations as a
 * device-side while loop, the mean-zero closure for pure-Neumann instances, the
 * true residual and the copy to x_i — is an independent branch.  hx_batch_solve
 * is then one graph launch and one synchronization for all instances, which
 * run concurrently on the GPU.  Not in the paper's method as such (it batches
 * its sub-problem solves).
 *   ops       host array of n operators (not owned; they must outlive the batch)
 *   b, x      host arrays of n device pointers (n_dof_i doubles each), bound at
 *             creation: the graph reads b_i and writes x_i on every solve
 *   rtol, max_it  stopping rule of every instance (as hx_solve_pcg, x0 = 0)
 *   lanes     number of chains the instances are spread over: instance i starts
 *             after instance i - lanes has finished, so at most `lanes` solves run
 *             side by side (0 or >= n: all instances concurrently).  Small
 *             instances gain from overlap; the many short kernels of multigrid
 *             V-cycles run better in few lanes.
 *             lanes = HX_BATCH_FUSED: lock-step mode.  The instances with a diagonal
 *             preconditioner (Jacobi, collocated mass) iterate together in one
 *             device-side while loop whose body holds, per CG iteration, one
 *             element-kernel launch per distinct (order, quadrature, geometry mode)
 *             walking a work list of (instance, element block) tiles, and one launch
 *             each for the assembly with (p, Ap), the update and the direction
 *             walking (instance, vector chunk) tiles, every reduction finished per
 *             instance; finished instances drop out of the passes, and the loop ends
 *             when all are done.  Small instances then share the device instead of
 *             each paying its own launches.  Instances with an LOR preconditioner
 *             run as branches beside the loop.
 *             lanes = HX_BATCH_AUTO (or any other negative value): autotuned — the
 *             first hx_batch_solve times one solve of the whole batch for each of 1,
 *             2, 4, 8, ... and n lanes and the lock-step mode (CUDA events on the
 *             batch's stream), keeps the fastest graph and then solves as usual;
 *             neither lanes nor mode changes the results (each instance's arithmetic,
 *             reductions included, is that of its solo hx_solve_pcg, bit for bit),
 *             only their overlap.  hx_batch_lanes reports the choice.
 * The graph captures the operators' coefficients and preconditioners: after
 * hx_op_set_coefficients on an HX_GEOM_ONTHEFLY operator, or hx_op_set_preconditioner,
 * create the batch again.  Synchronous create.
 */
typedef struct hx_batch hx_batch;
#define HX_BATCH_AUTO (-1)
#define HX_BATCH_FUSED (-2)
HX_API hx_status hx_batch_create(int n, hx_op* const* ops, const double* const* b, double* const* x, double rtol,
                                 int max_it, int lanes, hx_batch** out);

/* Solve every instance (after the caller's prior work on `stream`); infos: host array of n
 * results or NULL.  Returns HX_OK when all converged, else the first failing status.
 * Synchronous. */
HX_API hx_status hx_batch_solve(hx_batch* batch, void* stream, hx_solve_info* infos);

/* The lane count the next hx_batch_solve runs with, or HX_BATCH_FUSED for the lock-step mode
 * (after autotuning, the chosen one; before the first solve of an autotuned batch, n).  0 for a
 * NULL batch. */
HX_API int hx_batch_lanes(const hx_batch* batch);

/* Frees the batch (not its operators or vectors); NULL is ignored. */
HX_API void hx_batch_destroy(hx_batch* batch);

/*
 * Arithmetic-throughput probe (not part of the paper's method): enqueues on `stream`
 * one kernel that runs `iters` steps of 16 independent FMA chains per thread, in FP64
 * (fp64 != 0) or FP32, over one wave of resident blocks of 256 threads (at most 8 per SM),
 * and stores in *flops (host)
 * the floating-point operations it performs (2 per FMA).  Timing the launch with CUDA
 * events gives the device's measured FMA rate: the denominator beside which the FP64
 * operator's roofline fraction is reported.  HX_ERR_ARG for iters < 1 or flops NULL.
 * Stream-ordered; allocates nothing.
 */
HX_API hx_status hx_probe_fma(int fp64, int64_t iters, void* stream, double* flops);

/*
 * Operator apply that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc.  Examples are code inside a framework whose pool allocator owns
 * all device memory (an allocation behind its back can fail or fragment the
 * pool), services that fix their device memory budget at start-up, and
 * latency-bound loops that cannot pay for the device synchronization
 * cudaMalloc / cudaFree bring.  hx_op_create allocates an element-vector
 * workspace; this call instead uses a fixed array in the library's static
 * device memory (HX_NOALLOC_MAX_EVEC doubles, 32 MiB, held by every GPU that
 * loads the library until the process exits) and takes everything else from
 * the caller.
 *
 * Computes y = A x for A = alpha M + K(nu) with constant alpha, nu, geometric
 * factors recomputed from the element vertices (as HX_GEOM_ONTHEFLY), and no
 * Dirichlet elimination (the unconstrained operator of hx_op_apply).
 *   p, q        1 <= p <= 8, q in {p+1, p+2}
 *   n_elem      elements; n_elem (p+1)^3 must not exceed HX_NOALLOC_MAX_EVEC
 *               (else HX_ERR_UNSUPPORTED with a message saying so)
 *   n_dof       length of x and y
 *   X8          device, n_elem x 8 x 3 doubles: element corner coordinates,
 *               corner order c = cx + 2 cy + 4 cz
 *   restriction device, n_elem x (p+1)^3 int32 global DoF ids in [0, n_dof),
 *               local node order lexicographic (as hx_mesh_create)
 *   t_offsets   device, n_dof + 1 int32: the transpose of the restriction in
 *   t_indices   device, n_elem (p+1)^3 int32  compressed form: DoF g owns the
 *               positions t_indices[t_offsets[g] .. t_offsets[g+1]), each
 *               position e (p+1)^3 + l naming local node l of element e; the
 *               sum over them runs in the order given (increasing positions
 *               reproduce hx_op_apply bit for bit)
 *   x, y        device, n_dof doubles, not overlapping
 *   stream      stream the two kernels are enqueued on
 * The first call on a device (and again the first call in any other CUDA
 * context made current on it, e.g. after a device reset) looks up the scratch
 * array's device address (cudaGetSymbolAddress) with that device current and
 * caches it for that context; make that first call before capturing any
 * stream.  Every call on a device shares the
 * one scratch array and leaves its contents behind; the element kernel
 * overwrites every entry it later reads, so nothing needs clearing, but calls
 * whose work overlaps on the GPU (different streams, or several threads) race
 * on the array and must be serialized by the caller.  No device memory is
 * allocated or freed.  Stream-ordered.
 */
#define HX_NOALLOC_MAX_EVEC (1LL << 22)
HX_API hx_status hx_apply_noalloc(int p, int q, int64_t n_elem, int64_t n_dof, const double* X8,
                                  const int32_t* restriction, const int32_t* t_offsets, const int32_t* t_indices,
                                  double alpha, double nu, const double* x, double* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HX_H */
