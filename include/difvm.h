/*
 * difvm.h -- C ABI of the B300 (sm_103a) face-operator / PISO library.
 *
 * The operations follow the finite-volume method as a message-passing graph of
 * arxiv 2603.15920 ("DiFVM"):  cells are nodes, internal faces are edges
 * owner -> neighbour, boundary faces are edges from ghost nodes (Sec. 2.4.1).
 * Every operator computes a per-face message and reduces it onto cells with
 * sigma = +1 for the owner and -1 for the neighbour (Eq. aggregate).  The
 * reduction is a deterministic cell-CSR segmented sum in ascending face id:
 * no atomics, bitwise reproducible run to run.
 *
 * Conventions shared by all calls
 *  - Numbering.  difvm_mesh_create renumbers cells (reverse Cuthill-McKee) and
 *    faces (internal faces oriented owner < neighbour and sorted by
 *    (owner, neighbour); boundary faces kept grouped by patch, in patch order,
 *    sorted by owner inside a patch).  All field pointers below are in this
 *    INTERNAL numbering; difvm_mesh_permutation returns the maps.
 *  - Layout.  Cell fields are component-major  x[c * n_cells + i]  (SoA).
 *    Face fields  m[f], f < n_faces.  Boundary values  xb[c * n_boundary + b],
 *    b = f - n_internal.  Gradients  g[(c*3 + d) * n_cells + i] = d x_c / d x_d.
 *  - Precision.  prec selects the element type of every field pointer of the
 *    call: DIFVM_F64 (double) or DIFVM_F32 (float).  Krylov inner products and
 *    norms are always accumulated in double.
 *  - Memory.  Field pointers are DEVICE pointers owned by the caller; the
 *    library never frees them.  The mesh handle owns its own device copies of
 *    the geometry.  Hot calls allocate nothing (workspace comes from the caller
 *    or from a handle created beforehand) and are asynchronous on `stream`
 *    (a cudaStream_t; NULL = legacy default stream).
 *  - Errors.  Every call returns a difvm_status.  Argument and mesh errors are
 *    returned synchronously (nothing is launched); solver outcomes (not
 *    converged, breakdown, non-finite residual) are written to device-resident
 *    info structs so that calls never synchronise.  difvm_last_error() gives a
 *    thread-local message for the last non-OK status of the calling thread.
 */
#ifndef DIFVM_H
#define DIFVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DIFVM_OK = 0,
  DIFVM_EINVAL = 1,     /* bad argument or mesh */
  DIFVM_ENOMEM = 2,     /* device or host allocation failed (create calls only) */
  DIFVM_ECUDA = 3,      /* a CUDA runtime call failed */
  DIFVM_ENOTCONV = 4,   /* Krylov solve hit max_iter before the tolerance */
  DIFVM_EBREAKDOWN = 5, /* BiCGStab breakdown (rho or omega exactly 0) */
  DIFVM_ENONFINITE = 6, /* NaN / Inf residual */
  DIFVM_ETIMEOUT = 7    /* a bounded device wait gave up */
} difvm_status;

typedef enum { DIFVM_F32 = 0, DIFVM_F64 = 1 } difvm_prec;

/* Patch types of difvm_mesh_desc.patch_type (boundary conditions, Sec. 2.6.2):
 *   WALL   fixed velocity (value per face), zero-gradient pressure  (no-slip or moving wall)
 *   INLET  fixed velocity, zero-gradient pressure
 *   OUTLET zero-gradient velocity, fixed pressure (also the Windkessel outlet, Sec. 2.6.3)
 *   EMPTY  excluded from every face sum (2D runs) */
enum { DIFVM_PATCH_WALL = 0, DIFVM_PATCH_INLET = 1, DIFVM_PATCH_OUTLET = 2, DIFVM_PATCH_EMPTY = 3 };

/* Boundary-condition class of a field, chosen per operator call.  A class maps
 * every patch to one of FIXED (face value = the boundary value passed in),
 * ZEROGRAD (face value = owner cell value) or EMPTY (face skipped).
 *   VELOCITY  derived from patch types: WALL/INLET fixed, OUTLET zero-gradient
 *   PRESSURE  derived from patch types: OUTLET fixed, WALL/INLET zero-gradient
 *   ALL_FIXED / ALL_ZEROGRAD  every non-empty patch fixed / zero-gradient */
enum { DIFVM_BC_VELOCITY = 0, DIFVM_BC_PRESSURE = 1, DIFVM_BC_ALL_FIXED = 2, DIFVM_BC_ALL_ZEROGRAD = 3 };
enum { DIFVM_FACE_FIXED = 0, DIFVM_FACE_ZEROGRAD = 1, DIFVM_FACE_EMPTY = 2 };

enum { DIFVM_DIV_UPWIND = 0, DIFVM_DIV_LINEAR = 1 };           /* Eq. upwind / central */
enum { DIFVM_WK_EXACT = 0, DIFVM_WK_FE = 1, DIFVM_WK_BE = 2 };  /* Eq. windkessel_discrete */
enum { DIFVM_PCG = 0, DIFVM_BICGSTAB = 1 };
/* DIFVM_PRECOND_AMG: one V-cycle of aggregation multigrid per CG iteration
 * (pairwise aggregation on c_f, two passes per level, down to <= 192 cells;
 * Galerkin coarse operators summed in a fixed order every solve; two Jacobi
 * sweeps with degree-2 Chebyshev weights on [1/2, 2] (0.56, 1.39) before and
 * after the coarse correction, which is
 * scaled by 1.9; dense inverse on the coarsest level).  A fixed SPD operator:
 * it changes the iteration count, not the solution.  The paper uses ILU, whose
 * triangular solves are sequential along the mesh ordering.  Single-RHS CG on
 * a symmetric matrix only (EINVAL otherwise); the hierarchy is built on the
 * host on first use and kept by the mesh.  On a batched mesh the hierarchy is
 * built on the disjoint union (an aggregate never spans two cases, so each
 * case gets its own V-cycle) and every case keeps its own CG scalars and
 * stopping test; FP64 refinement is not available there (EINVAL), and EINVAL
 * too if the union does not coarsen to <= 192 cells (e.g. more than 192 cases). */
/* DIFVM_PRECOND_AMG_REUSE: as AMG, reusing the coefficient copy and multigrid
 * operators that the previous AMG solve with the same workspace built; the
 * caller guarantees the matrix is unchanged (e.g. the pressure matrix of the
 * second PISO corrector, which depends only on V/D). */
/* DIFVM_PRECOND_DIC: the incomplete factorisation the paper names (Sec. 2.6.1),
 * cells eliminated in the internal (RCM) numbering.  With CG on a symmetric
 * matrix: diagonal incomplete Cholesky, d_i = D_i - sum_{f: N(f)=i} L_f^2 /
 * d_O(f), M = (Dd + Lo) Dd^-1 (Dd + Lo^T).  With BiCGStab (1..3 right-hand
 * sides, e.g. the PISO momentum solve): diagonal incomplete LU of the
 * non-symmetric matrix, d_i = D_i - sum_{f: N(f)=i} L_f U_f / d_O(f),
 * M = (Dd + Lo) Dd^-1 (Dd + Up), right preconditioning.  Either way M = A on the
 * diagonal and on A's pattern.  The factor and each triangular sweep are one
 * launch whose rows wait (bounded) on the rows they depend on, level by level
 * (levels built on the host on first use and kept by the mesh; 437 on a 64^3
 * Kuhn mesh), so an application is a chain of that many dependent steps; a
 * wait that runs out ends the solve with DIFVM_ETIMEOUT.  Provided for fidelity
 * and comparison.  A single mesh only; FP32 or FP64 without refinement
 * (EINVAL otherwise). */
enum { DIFVM_PRECOND_NONE = 0, DIFVM_PRECOND_JACOBI = 1, DIFVM_PRECOND_AMG = 2,
       DIFVM_PRECOND_AMG_REUSE = 3, DIFVM_PRECOND_DIC = 4 };
enum { DIFVM_RENUMBER_RCM = 1u, DIFVM_SORT_FACES = 2u };
/* Index layouts of the face operators and solvers.  Where the (renumbered)
 * mesh allows it, a cell's half-face slots are 4-byte words holding both the
 * other cell and the face id as offsets (|j - i| < 2^14, face id within 2^15 of
 * the slice's first owned face), and the uniform width-4 ELL of the solvers
 * also keeps its columns as 16-bit offsets from the row (|j - i| < 2^15); else
 * the 8-byte (word, face id) slots and 32-bit columns are used.  The flag
 * DIFVM_WIDE_INDICES selects the wide layouts on any mesh (same results; for
 * testing both forms on small meshes). */
enum { DIFVM_WIDE_INDICES = 16u };
/* Split S_f = Delta_f + k_f of the diffusive flux (Eq. nonortho_flux, Sec. 2.3.2),
 * Delta_f along the cell-to-cell vector d, in bits 2-3 of the mesh flags:
 *   OVERRELAXED (0, the paper's default)  Delta = (|S| / |S^.d^|) d^
 *   MINIMUM                               Delta = (S.d^) d^
 *   ORTHOGONAL                            Delta = |S| d^
 *   NONE                                  the two-point flux |S| (phi_N - phi_O) / |d|, k = 0
 * It sets c_f = |Delta|/|d| and k_f = S - Delta for every operator, solver and
 * PISO step on the mesh.  Boundary faces (no d_ij) use |S|^2 / (S.d) with
 * d = x_f - C_O and no correction, for every split. */
enum { DIFVM_NONORTH_OVERRELAXED = 0u, DIFVM_NONORTH_MINIMUM = 4u, DIFVM_NONORTH_ORTHOGONAL = 8u,
       DIFVM_NONORTH_NONE = 12u, DIFVM_NONORTH_MASK = 12u };
enum { DIFVM_NONORTH_MOMENTUM = 1, DIFVM_NONORTH_PRESSURE = 2, DIFVM_NONORTH_ALL = 3 };

typedef struct difvm_mesh* difvm_mesh_t;

/* Mesh description (Sec. 2.4.1, static graph arrays).  All HOST pointers,
 * FP64 geometry, read during difvm_mesh_create only (copied).
 *   owner[n_faces], neighbour[n_internal]: cell ids; internal faces first,
 *     then boundary faces grouped by patch (patch p covers faces
 *     [patch_start[p], patch_start[p] + patch_size[p]) ).
 *   Sf[3*n_faces]: face area vector, AoS xyz, pointing out of the owner.
 *   Cf[3*n_faces]: face centroid.  V[n_cells]: volume.  C[3*n_cells]: centroid.
 *   n_cases / case_cell_start[n_cases+1]: a batch of independent meshes laid
 *     out as one disjoint union (cells of case k in [start[k], start[k+1]));
 *     no face may couple two cases.  A non-NULL case table (also with
 *     n_cases = 1) makes the mesh BATCHED: its Krylov solves are segmented,
 *     every case keeping its own scalars, convergence flag and iteration count
 *     (the result of a case does not depend on the other cases of the batch,
 *     bit for bit).  NULL for a single mesh (the single-mesh solvers).
 *   flags: DIFVM_RENUMBER_RCM | DIFVM_SORT_FACES (internal faces are always
 *     re-oriented so that owner < neighbour) | one DIFVM_NONORTH_* split |
 *     DIFVM_WIDE_INDICES (optional).
 *   device: CUDA device ordinal the handle lives on. */
typedef struct {
  int32_t n_cells, n_internal, n_faces, n_patches;
  const int32_t *owner, *neighbour;
  const double *Sf, *Cf, *V, *C;
  const int32_t *patch_start, *patch_size, *patch_type;
  int32_t n_cases;
  const int32_t *case_cell_start;
  uint32_t flags;
  int32_t device;
} difvm_mesh_desc;

/* Validate, renumber, build the cell-CSR and the derived face coefficients
 * (w_f, c_f = |Delta_f|/|d| (|S|^2/(S.d) for the default split), k_f = S - c_f d,
 * 1/V; Sec. 2.3.2) and upload them.
 * Errors: EINVAL with a message for index out of range, owner == neighbour,
 * patches not covering the boundary faces contiguously, V <= 0 or S.d <= 0,
 * more than 2^29 - 1 boundary faces; ENOMEM / ECUDA on allocation or copy
 * failure.  Synchronous. */
difvm_status difvm_mesh_create(const difvm_mesh_desc* desc, difvm_mesh_t* out);
/* Launch variants of the face operators (difvm_grad_gauss, difvm_div_flux,
 * difvm_laplacian, difvm_laplacian_apply) in FP32 on meshes whose rows all have
 * four faces (tetrahedra): the first call of each (operator, scheme or
 * correction, components) on a mesh times the variants -- register budgets
 * for 1, 6 and 8 resident 256-thread blocks per SM; the Gauss gradient's
 * second variant instead reads its face records by face id -- on that call's own
 * arguments and keeps the fastest for the mesh (the default unless another is
 * at least 2% faster).  That first call synchronises
 * with the host; a first call under stream capture launches the default
 * variant and records nothing.  No device memory is allocated.
 * The multigrid preconditioner's launch shapes are tuned once, when its
 * hierarchy is built (at the first call that needs it: a workspace query,
 * difvm_piso_create or a solve): per level below the mesh level, the lanes per
 * row of its sweeps (2, 4, 8) and per aggregate of its restriction (1, 8), by
 * timing whole V-cycles on a temporary workspace (allocated and freed then)
 * one level at a time; a shape replaces the default only if the V-cycle is at
 * least 2% faster.
 * mode 0: no timing, every call launches the default variant and the multigrid
 * takes its default shapes back; 1: timing on (the default); 2: forget the kept
 * choices and time again (the multigrid shapes at once).  Graphs already
 * captured keep the shapes they were captured with.  EINVAL on a bad mode. */
difvm_status difvm_mesh_autotune(difvm_mesh_t, int mode);
/* The kept choices, HOST outputs: keys[k] = operator << 8 | option << 4 |
 * components (operator 1 Gauss gradient, 2 divergence (option 1 upwind),
 * 3 Laplacian (option 1 with the non-orthogonal term), 4 LDU apply) and
 * variants[k] in 0..2; multigrid: operator 5 (option = level) with the lanes
 * per row, operator 6 (option = level) with the restriction's lanes per
 * aggregate; at most cap entries are written, *count gets the number kept. */
difvm_status difvm_mesh_tuning(difvm_mesh_t, uint32_t* keys, int32_t* variants, int cap, int32_t* count);
/* Multigrid V-cycle launch shape (DIFVM_PRECOND_AMG): levels of fewer than
 * tail_rows rows, and the coarsest dense solve, run as one cooperative kernel
 * (phases separated by grid barriers whose waits are bounded; a wait that runs
 * out ends the solve with DIFVM_ETIMEOUT) of tail_bps blocks per SM, instead
 * of five kernels per level; 0 rows: every level its own kernels.  -1 keeps
 * the library's choice (0 rows: on the B300 the per-level kernels, chained by
 * programmatic dependent launch, were faster; 2 blocks per SM).  Both forms
 * compute the same sums in the same order.  Takes effect at the next solve
 * that builds the multigrid operators.  EINVAL on tail_rows < -1 or tail_bps
 * 0 / < -1. */
difvm_status difvm_mesh_amg_config(difvm_mesh_t, int tail_rows, int tail_bps);
/* Maps between input and internal numbering, HOST outputs (any may be NULL):
 *   cell_new_of_old[n_cells], face_old_of_new[n_faces],
 *   face_flip[n_faces] (1 where the internal face was re-oriented: its S, and
 *   every face flux, changes sign). */
difvm_status difvm_mesh_permutation(difvm_mesh_t, int32_t* cell_new_of_old,
                                    int32_t* face_old_of_new, int8_t* face_flip);
/* Sizes: n_cells, n_internal, n_faces, n_boundary, n_patches, csr_entries. */
difvm_status difvm_mesh_info(difvm_mesh_t, int64_t out[6]);
/* Index layouts in use (see DIFVM_WIDE_INDICES), HOST output: out[0] = 1 if
 * the face operators read the 4-byte compact slot words, out[1] = 1 if the
 * solvers read 16-bit ELL column offsets (0: the wide forms). */
difvm_status difvm_mesh_layout(difvm_mesh_t, int32_t out[2]);
void difvm_mesh_destroy(difvm_mesh_t);

/* Geometry of a polyhedral mesh given by its vertices (the form of an OpenFOAM
 * polyMesh), producing the Sf, Cf, V, C of difvm_mesh_desc (Sec. 2.4.1 static
 * graph arrays; every element type: tetrahedra, hexahedra, prisms, pyramids,
 * general polyhedra).  All HOST pointers, caller-owned; no device work.
 *   points[3*n_points] (xyz); face f has the vertices
 *   face_pts[face_ptr[f] .. face_ptr[f+1]-1] (n_faces+1 pointers, >= 3 vertices
 *   per face) ordered so that their right-hand normal points out of owner[f];
 *   faces [0, n_internal) are internal with neighbour[f].
 * Faces are split into triangles around their vertex average, cells into
 * pyramids around the average of their face centroids (exact for planar faces).
 * Outputs Sf[3*n_faces], Cf[3*n_faces], V[n_cells], C[3*n_cells].
 * Errors: EINVAL with a message for out-of-range indices, faces with fewer than
 * three vertices or zero area, cells with fewer than four faces, and cells of
 * non-positive volume (faces not oriented out of their owner). */
difvm_status difvm_polymesh_geometry(int32_t n_points, const double* points, int32_t n_faces,
                                     const int32_t* face_ptr, const int32_t* face_pts,
                                     int32_t n_cells, const int32_t* owner, int32_t n_internal,
                                     const int32_t* neighbour, double* Sf, double* Cf, double* V,
                                     double* C);
const char* difvm_last_error(void);
/* Number of kernels this library has launched on the calling process (all
 * devices).  For launch accounting in benchmarks. */
uint64_t difvm_launch_count(void);
/* Algorithmic bytes of the Krylov and multigrid kernels launched so far
 * (momentum BiCGStab, pressure CG, V-cycles and their set-up): every array a
 * kernel must read or write counted once at its logical size -- a matrix as its
 * faces (owner, neighbour, coefficient(s)) plus its diagonal -- regardless of
 * layout, padding, re-reads or caching.  Counted at launch, so kernels that
 * exit early after convergence still count; launches inside a CUDA graph count
 * once, when captured.  For roofline accounting in benchmarks. */
uint64_t difvm_alg_bytes(void);
/* Per-kernel device timing for benchmarks: while active, every launch of the
 * kernel named by `tag` is bracketed by a pair of CUDA events on its own
 * stream (at most max_launches pairs; later launches are not timed).
 * difvm_prof_stop synchronises on the recorded events and returns the summed
 * kernel time and the number of timed launches; difvm_prof_bytes (before
 * difvm_prof_stop) the summed algorithmic bytes of the timed launches (as
 * difvm_alg_bytes counts them; multigrid tags only, 0 otherwise).
 * Process-wide, one tag at a time, not thread-safe; start/stop allocate and
 * free the events. */
enum { DIFVM_PROF_PCG_SPMV = 1, DIFVM_PROF_PCG_UPDATE = 2, DIFVM_PROF_PCG_PUPDATE = 3,
       DIFVM_PROF_AMG_RESID = 4,  /* fine-level multigrid residual r - A y */
       DIFVM_PROF_AMG_POST1C = 5  /* coarse-level corrected smoothing sweeps of eight lanes per row */ };
difvm_status difvm_prof_start(int tag, int max_launches);
difvm_status difvm_prof_stop(double* total_ms, int64_t* launches);
uint64_t difvm_prof_bytes(void);
/* Phases of the PISO step (Sec. 2.4.2): the Windkessel update and boundary
 * values; the momentum assembly (gradients, face and cell coefficients); the
 * momentum solve; per corrector the pressure assembly (HbyA, face fluxes,
 * pressure matrix), the pressure solve and the flux and velocity correction.
 * difvm_piso_step marks each phase with an NVTX range named "difvm:<phase>"
 * (visible to tools that record NVTX).  While difvm_phase_prof_start is active
 * it also records a CUDA event at every phase boundary on the step's stream (at
 * most max_marks, 6 + 3 n_corr per step); difvm_phase_prof_stop synchronises
 * and returns the summed milliseconds per phase in ms[DIFVM_PHASE_COUNT] and
 * the number of steps.  Host-loop steps only: steps under stream capture
 * (difvm_piso_step_graph) record nothing.  Process-wide, not thread-safe. */
enum { DIFVM_PHASE_WINDKESSEL = 0, DIFVM_PHASE_MOMENTUM_ASSEMBLY = 1, DIFVM_PHASE_MOMENTUM_SOLVE = 2,
       DIFVM_PHASE_PRESSURE_ASSEMBLY = 3, DIFVM_PHASE_PRESSURE_SOLVE = 4, DIFVM_PHASE_CORRECTION = 5,
       DIFVM_PHASE_COUNT = 6 };
difvm_status difvm_phase_prof_start(int max_marks);
difvm_status difvm_phase_prof_stop(double* ms, int64_t* steps);

/* ---------------------------------------------------------------- operators */
/* Gauss gradient (Eq. gauss_green): grad_i = (1/V_i) sum_f sigma phi_f S_f,
 * phi_f linearly interpolated (owner weight w_f) on internal faces and given by
 * the bc class on boundary faces.  phi[ncomp][nc], phi_b[ncomp][nb] (may be NULL
 * when the class has no FIXED patch), grad[ncomp][3][nc] (overwritten).
 * ncomp in 1..3. */
difvm_status difvm_grad_gauss(difvm_mesh_t, difvm_prec, int bc_class, const void* phi,
                              const void* phi_b, int ncomp, void* grad, void* stream);
/* Adjoint of difvm_grad_gauss: phi_bar += G^T grad_bar, phi_b_bar += G_b^T grad_bar
 * (accumulates; phi_b_bar may be NULL). */
difvm_status difvm_grad_gauss_bwd(difvm_mesh_t, difvm_prec, int bc_class, const void* grad_bar,
                                  int ncomp, void* phi_bar, void* phi_b_bar, void* stream);

/* Convective flux divergence (Eqs. conv_face_flux, upwind):
 * out_i = sum_f sigma m_f phi_f, phi_f upwind (m_f >= 0 -> owner) or linear on
 * internal faces, the bc-class value on boundary faces.  m[nf], phi/out [ncomp][nc]. */
difvm_status difvm_div_flux(difvm_mesh_t, difvm_prec, int scheme, int bc_class,
                            const void* mflux, const void* phi, const void* phi_b, int ncomp,
                            void* out, void* stream);
/* Adjoint: mflux_bar += dout/dm^T out_bar, phi_bar += ..., phi_b_bar += ...
 * (accumulates; any output may be NULL). */
difvm_status difvm_div_flux_bwd(difvm_mesh_t, difvm_prec, int scheme, int bc_class,
                                const void* mflux, const void* phi, const void* phi_b, int ncomp,
                                const void* out_bar, void* mflux_bar, void* phi_bar,
                                void* phi_b_bar, void* stream);

/* Diffusive flux (Eq. nonortho_flux, over-relaxed):
 * out_i = sum_f sigma gamma [c_f (phi_N - phi_O) + (grad phi)_f . k_f], boundary
 * FIXED faces gamma c_f (phi_b - phi_O) (orthogonal), others 0.  grad may be NULL
 * (orthogonal part only); (grad phi)_f is linearly interpolated. */
difvm_status difvm_laplacian(difvm_mesh_t, difvm_prec, int bc_class, double gamma,
                             const void* phi, const void* phi_b, const void* grad, int ncomp,
                             void* out, void* stream);
/* Adjoint of difvm_laplacian w.r.t. phi, phi_b and grad (accumulates). */
difvm_status difvm_laplacian_bwd(difvm_mesh_t, difvm_prec, int bc_class, double gamma,
                                 const void* out_bar, int ncomp, void* phi_bar, void* phi_b_bar,
                                 void* grad_bar, void* stream);

/* Matrix-free LDU operator (Eq. Ap_H, the implicit momentum / pressure matrix):
 * y_i = D_i x_i + sum_{f: O(f)=i} U_f x_N(f) + sum_{f: N(f)=i} L_f x_O(f).
 * diag[nc], lower[ni], upper[ni] (NULL = symmetric, U = L); x, y [ncomp][nc].
 * transpose != 0 applies A^T (L and U swapped). */
difvm_status difvm_laplacian_apply(difvm_mesh_t, difvm_prec, const void* diag, const void* lower,
                                   const void* upper, const void* x, int ncomp, int transpose,
                                   void* y, void* stream);
/* Adjoint: x_bar += A^T y_bar; diag_bar_i += sum_c y_bar_i x_i;
 * lower_bar_f += sum_c y_bar_N x_O; upper_bar_f += sum_c y_bar_O x_N
 * (accumulates; any output may be NULL; with upper == NULL the symmetric
 * coefficient gets both contributions in lower_bar).  tmp: device scratch of
 * ncomp*n_cells elements, required when x_bar != NULL. */
difvm_status difvm_laplacian_apply_bwd(difvm_mesh_t, difvm_prec, const void* diag,
                                       const void* lower, const void* upper, const void* x,
                                       const void* y_bar, int ncomp, void* x_bar, void* diag_bar,
                                       void* lower_bar, void* upper_bar, void* tmp, void* stream);
/* Same adjoint as difvm_laplacian_apply_bwd, for callers that cannot allocate
 * device memory -- for example a host whose device memory is all owned by
 * another runtime's pool, or a time-critical loop in which a cudaMalloc (which
 * may synchronise the whole device) is not acceptable.  It takes no tmp
 * argument: A^T y_bar is formed in a 16 MiB scratch array built into the
 * library (every GPU that loads the library keeps it reserved until the process
 * exits).  The paper has no counterpart; this is a library convenience.
 * Limits and behaviour:
 *  - with x_bar != NULL, ncomp * n_cells * sizeof(element) must be at most
 *    16 MiB (FP64: 2,097,152 elements, FP32: 4,194,304); larger calls return
 *    EINVAL with a message and launch nothing;
 *  - the first call on a device looks up the array's device address with that
 *    device current; make that first call before any stream capture;
 *  - calls share the one array and it keeps the last call's contents (every
 *    element used is overwritten before it is read, so nothing needs
 *    clearing); each GPU has its own copy, and calls on the same GPU that
 *    can overlap (for example on two streams with no ordering between them)
 *    race on it;
 *  - the mesh's device must be the current device (EINVAL otherwise);
 *  - no cudaMalloc, cudaFree or allocating library routine is called. */
difvm_status difvm_laplacian_apply_bwd_noalloc(difvm_mesh_t, difvm_prec, const void* diag,
                                               const void* lower, const void* upper, const void* x,
                                               const void* y_bar, int ncomp, void* x_bar,
                                               void* diag_bar, void* lower_bar, void* upper_bar,
                                               void* stream);

/* ------------------------------------------------------------------- Krylov */
typedef struct {
  int32_t method;      /* DIFVM_PCG (SPD) or DIFVM_BICGSTAB */
  int32_t precond;     /* DIFVM_PRECOND_NONE, DIFVM_PRECOND_JACOBI or DIFVM_PRECOND_AMG */
  int32_t max_iter;
  int32_t check_every; /* iterations between host convergence checks (0 = 8) */
  double tol_rel;      /* stop when ||b - A x||_2 <= max(tol_rel ||b||_2, tol_abs) */
  double tol_abs;
  int32_t refine_max;  /* refinement sweeps (difvm_krylov_solve_refine; in PISO a value > 0
                          with DIFVM_F32 selects the mixed-precision pressure solve) */
  double inner_tol;    /* refinement: relative tolerance of each inner F32 solve (0 = 1e-4) */
} difvm_solve_opts;

/* Per-component outcome, written on the DEVICE (no host sync needed). */
typedef struct {
  int32_t iters, refinements, status, pad;
  double res0, res, bnorm;
} difvm_solve_info;

/* Bytes of workspace a solve with these options needs: difvm_krylov_solve and
 * difvm_krylov_solve_bwd, and also difvm_krylov_solve_refine when prec is F32
 * and opts->refine_max > 0; covers
 * the multigrid preconditioner (whose hierarchy this call builds on first use).
 * 0 for an invalid combination. */
size_t difvm_krylov_opts_workspace_bytes(difvm_mesh_t, difvm_prec, const difvm_solve_opts* opts,
                                         int ncomp);
/* Bytes of workspace difvm_krylov_solve needs for (prec, method, ncomp) with
 * Jacobi or no preconditioning. */
size_t difvm_krylov_workspace_bytes(difvm_mesh_t, difvm_prec, int method, int ncomp);
/* Solve A x_c = b_c for each of ncomp right-hand sides with the LDU matrix
 * (diag, lower, upper; upper NULL = symmetric) by Jacobi-preconditioned CG or
 * BiCGStab (Sec. 2.6.1: CG for the SPD pressure system, BiCGStab for the
 * momentum system).  x is the initial guess on entry and the solution on exit.
 * Inner products and norms are accumulated in FP64.  info_dev[ncomp] is device
 * memory; on a batched mesh info_dev[n_cases * ncomp], case-major, and each
 * case stops on its own residual.  The call synchronises `stream` every check_every iterations to read
 * the convergence flags (iterations issued past convergence do nothing).
 * Returns OK or the worst solver status (ENOTCONV, EBREAKDOWN, ENONFINITE);
 * x holds the last iterate in every case. */
difvm_status difvm_krylov_solve(difvm_mesh_t, difvm_prec, const difvm_solve_opts* opts,
                                const void* diag, const void* lower, const void* upper,
                                const void* b, void* x, int ncomp, void* workspace,
                                size_t workspace_bytes, difvm_solve_info* info_dev, void* stream);
/* Bytes of workspace difvm_krylov_solve_refine needs. */
size_t difvm_krylov_refine_workspace_bytes(difvm_mesh_t, int method, int ncomp);
/* Mixed-precision solve with iterative refinement: the matrix is FP32
 * (diag/lower/upper float), b64 and x64 are FP64.  Each sweep forms the FP64
 * residual r = b - A x (FP32 coefficients are exact in FP64), solves A e = r in
 * FP32 to opts->inner_tol (relative, 0 = 1e-4) and adds e to x64 in FP64, until
 * ||r||_2 <= max(tol_rel ||b||_2, tol_abs) or refine_max sweeps (0 = 20); a
 * sweep that fails to cut the residual by 4x stops with ENOTCONV.
 * info.iters = total inner iterations, info.refinements = sweeps.  With
 * DIFVM_PRECOND_AMG the solve is instead one CG in FP64 (x, r, p, q, inner
 * products; FP32 coefficients) preconditioned by the FP32 V-cycle: it reaches
 * the FP64 tolerance without sweeps (refine_max and inner_tol are not used,
 * info.refinements = 0).  EINVAL on batched meshes. */
difvm_status difvm_krylov_solve_refine(difvm_mesh_t, const difvm_solve_opts* opts, const float* diag,
                                       const float* lower, const float* upper, const double* b64,
                                       double* x64, int ncomp, void* workspace,
                                       size_t workspace_bytes, difvm_solve_info* info_dev,
                                       void* stream);
/* Adjoint of a converged solve (implicit differentiation, Eq. implicit_diff):
 * b_bar_c = A^{-T} x_bar_c (same method on the transposed matrix), then
 * diag_bar_i -= sum_c b_bar_i x_i, lower_bar_f -= sum_c b_bar_N x_O,
 * upper_bar_f -= sum_c b_bar_O x_N.  b_bar is OVERWRITTEN with A^{-T} x_bar
 * (the caller accumulates it where needed); coefficient grads accumulate. */
difvm_status difvm_krylov_solve_bwd(difvm_mesh_t, difvm_prec, const difvm_solve_opts* opts,
                                    const void* diag, const void* lower, const void* upper,
                                    const void* x, const void* x_bar, int ncomp, void* b_bar,
                                    void* diag_bar, void* lower_bar, void* upper_bar,
                                    void* workspace, size_t workspace_bytes,
                                    difvm_solve_info* info_dev, void* stream);

/* --------------------------------------------------------------- Windkessel */
/* One RCR step per outlet (Eqs. windkessel_ode, windkessel_discrete), all
 * DEVICE double arrays [n_out]:  EXACT  p_c <- p_c e + R_d Q (1-e), e = exp(-dt/(R_d C));
 * FE  p_c <- p_c + dt (Q - p_c/R_d)/C;  BE  p_c <- (p_c + dt Q/C)/(1 + dt/(R_d C));
 * then p_out = p_c + R_p Q.  pc is updated in place. */
difvm_status difvm_windkessel_update(int n_out, int scheme, const double* Rp, const double* C,
                                     const double* Rd, const double* Q, double dt, double* pc,
                                     double* p_out, void* stream);
/* Adjoint of one step given the inputs (pc_in = p_c before the step):
 * from pc_out_bar, p_out_bar accumulate pc_in_bar, Q_bar, Rp_bar, C_bar, Rd_bar
 * (device double [n_out]; pc_in_bar is overwritten, the others accumulate). */
difvm_status difvm_windkessel_update_bwd(int n_out, int scheme, const double* Rp, const double* C,
                                         const double* Rd, const double* Q, double dt,
                                         const double* pc_in, const double* pc_out_bar,
                                         const double* p_out_bar, double* pc_in_bar, double* Q_bar,
                                         double* Rp_bar, double* C_bar, double* Rd_bar, void* stream);

/* --------------------------------------------------------------------- PISO */
typedef struct {
  double nu, dt;
  int32_t n_corr;       /* pressure correctors (Sec. 2.4.2: typically 2) */
  int32_t nonorth;      /* explicit over-relaxed non-orthogonal corrections, bitmask of
                           DIFVM_NONORTH_MOMENTUM (momentum diffusion) and
                           DIFVM_NONORTH_PRESSURE (pressure Laplacian, lagged); 0 = none */
  difvm_solve_opts solve_U, solve_p;
  int32_t pref_cell;    /* internal id of the pinned cell when no patch fixes p; on a
                           batched mesh relative to each case's first cell, for every
                           case with no fixed-pressure face */
  int32_t wk_scheme;    /* DIFVM_WK_* */
  int32_t n_out;        /* Windkessel outlets (0..16) */
  int32_t wk_patch[16]; /* patch ids of the outlets */
  double nonorth_limit; /* psi in (0,1): cap each explicit non-orthogonal correction at
                           psi/(1-psi) x the face's orthogonal part (the "limited" form of
                           Eq. nonortho_flux); 0 or >= 1: unlimited over-relaxed correction */
  int32_t conv;         /* momentum convection: DIFVM_CONV_UPWIND (Eq. upwind, implicit) or
                           DIFVM_CONV_SOU, second-order upwind by deferred correction (Eqs.
                           deferred_correction, sou): the matrix stays upwind and each internal
                           face adds m_f (grad U^n)_C . (x_f - x_C) of its upwind cell C to the
                           explicit part (boundary faces keep their condition's face value) */
  int32_t time_scheme;  /* momentum predictor: DIFVM_TIME_BE (backward Euler) or DIFVM_TIME_CN
                           (Crank-Nicolson: the convection-diffusion operator A and its source b
                           averaged over the two time levels, (V/dt + A/2) U* = V/dt U^n + b -
                           A U^n / 2, the face flux and the explicit corrections from step n) */
} difvm_piso_opts;
enum { DIFVM_CONV_UPWIND = 0, DIFVM_CONV_SOU = 1 };
enum { DIFVM_TIME_BE = 0, DIFVM_TIME_CN = 1 };

typedef struct difvm_piso* difvm_piso_t;
/* Create a PISO driver for one mesh and precision; owns all step workspace. */
difvm_status difvm_piso_create(difvm_mesh_t, difvm_prec, const difvm_piso_opts*, difvm_piso_t*);
void difvm_piso_destroy(difvm_piso_t);
/* Per-step outcome (device): solver iterations and the Windkessel values. */
typedef struct {
  int32_t itU[3], itp[4], status, pad;
  double Q[16], p_out[16];
} difvm_piso_info;
/* One PISO step (Sec. 2.4.2), in place on U[3][nc], p[nc], phi[nf]:
 *  1. Windkessel outlets: Q_o = sum over the patch of phi, p_c update,
 *     p_out = p_c + R_p Q imposed as the fixed pressure of the patch (p_b);
 *  2. momentum predictor: backward Euler, implicit upwind convection with the
 *     current phi, implicit orthogonal + explicit non-orthogonal diffusion,
 *     A U* = b - V grad p^n, BiCGStab per component;
 *  3. n_corr times: HbyA = (b - offdiag U)/D, phiHbyA_f = HbyA_f.S_f, pressure
 *     equation with face coefficient (V/D)_f c_f (PCG), Rhie-Chow flux
 *     correction phi = phiHbyA - (V/D)_f (c_f dp + (grad p)_f.k_f), velocity
 *     correction U = HbyA - (V/D) grad p.
 * U_b[3][nb], p_b[nb] boundary values at the new time level (p_b is rewritten
 * on Windkessel patches); wk: DEVICE double [4*n_out] = (Rp, C, Rd, p_c) with
 * p_c updated; info_dev device.  All device pointers of the handle's precision
 * except wk (double).  Synchronises on Krylov convergence checks. */
difvm_status difvm_piso_step(difvm_piso_t, void* U, void* p, void* phi, const void* U_b, void* p_b,
                             double* wk, difvm_piso_info* info_dev, void* stream);

/* ------------------------------------------------------ adjoint of a step */
/* Reverse-mode derivative of one PISO step (Sec. 2.5, Eq. vjp), written by hand
 * stage by stage; the two linear solves are differentiated implicitly
 * (Eq. implicit_diff): for x = A^{-1} r, r_bar = A^{-T} x_bar solved by the
 * step's own Krylov method and settings on A^T, and A_bar = -r_bar x^T.
 * Non-smooth switches (upwind max(m,0), the limiter of nonorth_limit) take the
 * derivative of the branch the forward step took.
 *
 * Tape: device memory the caller owns, at least difvm_piso_tape_bytes(h) bytes,
 * 256-byte aligned.  difvm_piso_step_record is difvm_piso_step (same arguments,
 * same results, bit for bit) that also writes into the tape what the reverse
 * sweep needs: the step's input U, p, phi, p_b after the Windkessel update, the
 * capacitor pressures before it and the outlet flows, the predicted velocity
 * and every corrector's U and p.  A tape belongs to the handle that wrote it. */
size_t difvm_piso_tape_bytes(difvm_piso_t);
difvm_status difvm_piso_step_record(difvm_piso_t, void* U, void* p, void* phi, const void* U_b,
                                    void* p_b, double* wk, difvm_piso_info* info_dev, void* tape,
                                    size_t tape_bytes, void* stream);
/* Adjoint of the recorded step.  U_b and wk (its R_p, C, R_d) must be the
 * values the recorded step used.  In place, like the forward step:
 *   U_bar[3][nc], p_bar[nc], phi_bar[nf], p_b_bar[nb] hold on entry the
 *   adjoints of the step's outputs U, p, phi, p_b and on return those of its
 *   inputs (p_b_bar may be NULL: zero on entry, not returned); on Windkessel
 *   patches the input p_b is overwritten by the step, so its adjoint is 0;
 *   wk_bar: DEVICE double [4*n_out]; entries 0..2 (R_p, C, R_d) accumulate,
 *   entry 3 holds the adjoint of p_c after the step on entry and before it on
 *   return (NULL allowed without outlets).
 * Accumulated: U_b_bar[3][nb] (may be NULL), *nu_bar (device double, may be
 * NULL; a fixed-order FP64 sum).  info_dev (may be NULL): itU = iterations of
 * the transposed momentum solve, itp = those of each corrector's adjoint
 * pressure solve, Q = the outlet-flow adjoints, p_out = the outlet-pressure
 * adjoints.  Field pointers are of the handle's precision.  The first call
 * allocates the adjoint workspace (about 30 x nc + 10 x n_internal values);
 * the handle's forward workspace is reused, so a forward step and a
 * backward step must not run concurrently on one handle.  Every sum has a
 * fixed order: results are bitwise reproducible.  Returns OK or the worst
 * status of the adjoint solves; EINVAL for a short or misaligned tape.
 * Each adjoint solve starts from the handle's solution of the same solve in
 * the previous call (the reverse-time analogue of the forward step starting
 * from p^n); the result then depends on the call sequence only within the
 * solver tolerance.  difvm_piso_adjoint_reset zeroes those starting guesses
 * (the first call after create starts from zero). */
difvm_status difvm_piso_step_bwd(difvm_piso_t, const void* tape, size_t tape_bytes,
                                 const void* U_b, const double* wk, void* U_bar, void* p_bar,
                                 void* phi_bar, void* p_b_bar, double* wk_bar, void* U_b_bar,
                                 double* nu_bar, difvm_piso_info* info_dev, void* stream);
difvm_status difvm_piso_adjoint_reset(difvm_piso_t, void* stream);
/* The same step as a CUDA graph: on the first call for an argument set
 * (U, p, phi, U_b, p_b, wk, info_dev) the step is captured on an internal
 * stream, every Krylov solve as a device-side conditional WHILE loop (a few
 * iterations per pass, a one-thread kernel setting the loop condition from the
 * solver state, bounded by max_iter), and instantiated; each call then
 * launches that graph on `stream` (one launch, no host synchronisation, no
 * host-side convergence checks).  Results equal difvm_piso_step's bit for bit
 * (iterations past convergence do nothing).  The outcome is only in info_dev
 * (required); the return value reports argument and launch errors.  The
 * handle keeps one graph per argument set until destroyed.  Not with
 * difvm_prof_start active. */
difvm_status difvm_piso_step_graph(difvm_piso_t, void* U, void* p, void* phi, const void* U_b,
                                   void* p_b, double* wk, difvm_piso_info* info_dev, void* stream);
/* Initial face flux phi_f = U_f . S_f (linear interpolation; boundary: U_b.S
 * for fixed velocity, U_O.S for zero gradient, 0 for empty). */
difvm_status difvm_flux_from_U(difvm_mesh_t, difvm_prec, const void* U, const void* U_b,
                               void* phi, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DIFVM_H */
