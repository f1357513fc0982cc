/*
 * vembddc -- BDDC-preconditioned CG for the divergence-free virtual element
 * discretization of the 3D Stokes equations, on one GPU (sm_103a).
 *
 * Method: T. Bevilacqua, F. Dassi, S. Zampini, S. Scacchi, "BDDC
 * preconditioners for virtual element approximations of the
 * three-dimensional Stokes equations".  Section, equation and table names
 * below refer to that paper.
 *
 * Conventions shared by every call
 * --------------------------------
 * Status: every call returns a vem_status (0 = success, < 0 = error); no call
 * aborts, traps or exits.  vem_last_error() returns a message for the last
 * failure in the calling thread.
 *
 * Pointers: "host" arrays are read during the call only and copied; the
 * library never keeps them.  "device" arrays are caller-owned CUDA device
 * memory (for example torch tensors) that must stay valid for the call; the
 * library works on the stream set with vem_set_stream (default: the legacy
 * default stream) and returns once its work on that stream is enqueued,
 * except where a call says it synchronizes.
 *
 * Global DOF order (Sec. 3, DOFs D1-D5; one number per velocity component):
 *   vertex v            : 3 v + c                                   (D1)
 *   edge e, point j     : nV*3 + (e*(k-1) + j)*3 + c                (D2)
 *   face f, monomial b  : off_f + (f*dim P_{k-2}(2D) + b)*3 + t     (D3)
 *   element K           : off_k + K*(n4+n5) + (D4 then D5)          (D4,D5)
 * with c = x,y,z; t = 0 normal, 1 first tangent, 2 second tangent.
 * Edges are numbered in order of first appearance when the face loops are
 * read face by face; edge points are the interior Gauss-Lobatto nodes,
 * ordered from the lower-numbered vertex.  Face frames: n = the face's
 * global normal (loop orientation), t1 = unit first loop edge, t2 = n x t1;
 * moments are averages (1/|f|) int over the face against the scaled
 * monomials of P_{k-2} in the face frame centred at the vertex average.
 * D4: averages (1/|K|) int v . (xi ^ m_b e_c), xi = (x - x_K)/h_K (x_K the
 * vertex average, h_K the diameter), b over P_{k-3} and c = x,y,z, graded
 * monomial order, minus the dependent generator (b = xi_3, c = z) at k = 4.
 * D5: averages (1/|K|) int div v m_a for the scaled monomials of degree
 * 1..k-1.  Pressure: per element, the coefficients of the scaled monomials
 * of P_{k-1}(K).  Vectors passed to the solver calls ("system vectors")
 * hold the free (non-Dirichlet) velocity DOFs in increasing global order,
 * then all element pressures (element-major).
 */
#ifndef VEMBDDC_H
#define VEMBDDC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VEM_OK = 0,
  VEM_EINVAL = -1,     /* bad argument (null pointer, size, mesh topology) */
  VEM_ENOMEM = -2,     /* device or host allocation failed */
  VEM_ECUDA = -3,      /* a CUDA call failed */
  VEM_ESINGULAR = -4,  /* zero or wrong-signed pivot in a local or coarse factorization */
  VEM_EBREAKDOWN = -5, /* CG breakdown (p^T S p <= 0 or a non-finite value) */
  VEM_ENOTCONV = -6,   /* CG reached maxit above rtol */
  VEM_ETIMEOUT = -7    /* a bounded device wait gave up */
} vem_status;

/* Polyhedral mesh (Sec. 3, "Mesh construction").  All host arrays.
 * Faces are planar vertex loops; a loop's orientation fixes the face's
 * global normal.  elem_face holds +(f+1) when the global normal of face f
 * points out of the element and -(f+1) otherwise. */
typedef struct {
  int32_t nV;
  const double* xyz;        /* [nV*3] */
  int32_t nF;
  const int32_t* face_ptr;  /* [nF+1] */
  const int32_t* face_vtx;  /* [face_ptr[nF]] */
  int32_t nE;
  const int32_t* elem_ptr;  /* [nE+1] */
  const int32_t* elem_face; /* [elem_ptr[nE]] signed, 1-based */
} vem_mesh;

typedef struct vem_system vem_system;
typedef struct bddc bddc;

/* Builds the VEM discretization of degree k (2 <= k <= 4) of the Stokes
 * problem with homogeneous Dirichlet velocity on the boundary (Eq.
 * DiscProblem): per-element projectors and local matrices on the GPU
 * (Eq. discreteA with nu_K as factor, B_K exact from the DOFs) and the global
 * CSR matrix K = [A B^T; B 0] over the free velocity DOFs and all element
 * pressures (Eq. MatrixForm).  nu_per_element: host [nE].  Synchronizes. */
int vem_assemble(const vem_mesh* mesh, int k, const double* nu_per_element, vem_system** out);

/* The reduced scheme (the remark after the convergence theorem, Sec. 3):
 * as vem_assemble, but the velocity is restricted to fields whose element
 * divergence moments of degree >= 1 vanish (every D5 DOF is eliminated like
 * a Dirichlet DOF, with value 0) and the pressure to one constant per
 * element (B keeps its first row, the face fluxes).  The full scheme's
 * velocity is divergence-free and therefore lies in this space, so the
 * velocity is the same; the system has nE * (2 dim P_{k-1} - 2) fewer
 * unknowns.  vem_dof_layout reports nE pressures; every other call works
 * unchanged on the reduced system. */
int vem_assemble_reduced(const vem_mesh* mesh, int k, const double* nu_per_element, vem_system** out);

/* Statistics by name: "nnz" (nonzeros of K), "n_elements", "reduced" (1 for
 * a system of vem_assemble_reduced), and the
 * vem_assemble phase wall times (host clock) "t_topology_ms" (topology, DOF
 * numbering, element records), "t_element_launch_ms" (uploads and the
 * element kernel launch), "t_pattern_ms" (CSR pattern on the host while the
 * element kernel runs), "t_element_wait_ms" (waiting for the element kernel
 * after that), "t_pattern_upload_ms" (pattern upload, assembly launch),
 * "t_gpu_finish_ms" (waiting for the GPU).  Unknown keys: VEM_EINVAL. */
int vem_info(const vem_system* sys, const char* key, double* value);

/* Sizes: free velocity DOFs, element pressures, all velocity DOFs. */
int vem_dof_layout(const vem_system* sys, int64_t* n_vel_free, int64_t* n_press, int64_t* n_vel_all);

/* Host copy of the map free-velocity index -> global velocity DOF number. */
int vem_free_dofs(const vem_system* sys, int64_t* free_to_global /* host [n_vel_free] */);

/* Quadrature points of the load rule of exactness `degree` (collapsed Gauss
 * product rule with (degree+3)/2+1 points per direction on each tetrahedron
 * (x_K, face fan triangle); point order: element, face, fan triangle, then
 * the rule's points).  With xyz_out == NULL only *n is set.  xyz_out: host
 * [n*3]. */
int vem_quad_points(vem_system* sys, int degree, int64_t* n, double* xyz_out);

/* Load vector (Eq. discreteF): rhs = [int Pi^0_k f . phi_i ; 0] over the
 * system vector layout, from f sampled at the points of vem_quad_points with
 * the same degree.  f_at_quad: [n*3], host memory (copied to the device in
 * the call) or device memory (read in place); rhs_dev: device
 * [n_free+n_press]. */
int vem_load(vem_system* sys, int degree, const double* f_at_quad, double* rhs_dev);

/* Non-homogeneous Dirichlet data for tests such as the polynomial patch test
 * (convergence theorem, Sec. 3: polynomial solutions of degree k are
 * reproduced exactly).  The system keeps the boundary velocity DOFs fixed and
 * eliminated; this call moves their prescribed values to the right-hand side
 * of the free saddle system (Eq. MatrixForm):
 *   f_dev[r] -= sum over fixed velocity DOFs j of K[r][j] g_host[j]
 * for every free velocity row and every pressure row r.
 * g_host: host [n_vel], values of ALL velocity DOFs in the global numbering
 * (vertex, edge, face, element-interior DOFs; only the fixed ones are read;
 * in the reduced scheme the eliminated D5 DOFs are fixed too and read as
 * their prescribed values, normally 0).  f_dev: device [n_free+n_press],
 * updated in place.  Allocates temporary device memory; synchronizes the
 * system's stream.  Errors: VEM_EINVAL on null arguments. */
int vem_lift_dirichlet(vem_system* sys, const double* g_host, double* f_dev);

/* Load vector without device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * themselves or through the library, for example code running under a
 * memory budget fixed in advance, or inside a framework that owns every
 * device allocation through its own pool.
 *
 * Computes the same vector as vem_load, but f is given on the device:
 * f_at_quad_dev: device [n*3], the load f sampled at the points of
 * vem_quad_points(sys, degree, ...) in that order; rhs_dev: device
 * [n_free+n_press], overwritten.  Neither is kept after the call.
 * Its only scratch is one fixed array of 16 MiB compiled into the library:
 * every GPU that loads the library holds it until the process exits.  It
 * holds the quadrature offsets ((nE+1) int64 values, padded to 256 bytes)
 * and the element load vectors (8 bytes per element velocity DOF);
 * a mesh that needs more returns VEM_EINVAL with the required size in
 * vem_last_error() and writes nothing (use vem_load there).
 * Calls no cudaMalloc, cudaFree or other allocating routine.  The work is
 * enqueued on the system's stream and the call returns without waiting.
 * Every call uses the same scratch array and every call rewrites what it
 * reads, so calls that run one after another on the GPU give independent
 * results; calls whose GPU work overlaps (other streams, other threads,
 * other handles on the same device) race on the array.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Call it with the system's device current. */
int vem_load_noalloc(vem_system* sys, int degree, const double* f_at_quad_dev, double* rhs_dev);

/* y = K x over the system vector layout (Eq. MatrixForm).  Device arrays. */
int vem_apply(vem_system* sys, const double* x_dev, double* y_dev);

/* Test access: copies the local matrices of `count` elements to the host.
 * A: [count * nK * nK] row-major (nK = velocity DOFs of the element, in
 * the order vertices (increasing), edges (increasing), faces (element
 * order), D4, D5); B: [count * nP * nK]; dofs: [count * nK] global velocity
 * numbers.  Elements must all have the same nK (returned in *nK). */
int vem_element_matrices(vem_system* sys, const int32_t* elems, int32_t count, int32_t* nK,
                         double* A, double* B, int64_t* dofs);

/* Test access: CSR of K (system layout).  With vals == NULL only sizes. */
int vem_csr(vem_system* sys, int64_t* n, int64_t* nnz, int64_t* row_ptr, int32_t* col, double* vals);

int vem_set_stream(vem_system* sys, void* cuda_stream);

/* Diagnostics: number of kernels the library has launched since it was
 * loaded (all handles, all threads). */
int vem_kernel_launches(int64_t* count);
void vem_free(vem_system* sys);
const char* vem_last_error(void);

/* ---------------------------------------------------------------- BDDC
 * Primal constraint set (Sec. 5.1), bit mask:                              */
#define BDDC_VERTEX 1u  /* all subdomain vertices primal                      */
#define BDDC_EDGE 2u    /* per macro edge: the three component means            */
#define BDDC_FACE 4u    /* per macro face: the three component integrals        */
#define BDDC_FLUX 8u    /* per macro face: the normal flux (Eq. primalfacen)     */
#define BDDC_ALL 16u    /* every interface DOF primal (test: M^{-1} = S^{-1})   */
/* scaling: averaging of the dual interface values (Sec. 4.3, Sec. 6)       */
#define BDDC_SCALING_MULTIPLICITY 0   /* 1/card on every dual DOF (Eq. pseudoinv)   */
#define BDDC_SCALING_DELUXE 1         /* deluxe on macro faces, 1/card on edges     */
#define BDDC_SCALING_DELUXE_EDGES 2   /* deluxe on macro faces and on macro edges:
                                         D_E^(k) = (sum_j S_E^(j))^-1 S_E^(k) over the
                                         subdomains j sharing the edge E (the face
                                         formula of Sec. 6 taken over card(E) >= 3
                                         subdomains instead of 1/card)              */

typedef struct {
  int32_t precision;        /* local factors and sweeps: 0 FP64; 1 FP32 with one step of
                               refinement per local solve (residual in FP64 from the
                               element matrices); 2 FP32 without refinement.  Coarse
                               matrix, deluxe inverses, operator and CG stay FP64. */
  int32_t scaling;          /* unused (the bddc_setup argument decides)        */
  uint32_t constraints;     /* unused (the bddc_setup argument decides)        */
  double adaptive_threshold;/* theta > 0 (deluxe scalings only): adaptive coarse
                               space of Sec. 6.  Per macro face, the generalized
                               eigenproblem (S~_i : S~_j) psi = lambda (S_i : S_j) psi
                               on the face's dual coordinates (S_s the face block of
                               the subdomain Schur complement, S~_s the Schur
                               complement of the constrained Neumann matrix onto
                               the face, A : B = (A^-1 + B^-1)^-1); every eigenvector
                               with lambda < 1/theta adds the primal functional
                               (S_i : S_j) psi, and the setup is run again with the
                               enlarged primal space (at most 64 per face).  0: off */
  int32_t nd_leaf;          /* elements per nested-dissection leaf (0: 4)      */
  int32_t use_graph;        /* 0 or 1: pcg_solve runs its whole loop as one CUDA
                               graph launch (a conditional while node whose body is
                               one iteration, scalars and stop rule on the device)
                               and bddc_apply replays a captured graph (captured
                               again when r or z change); -1: host-driven loop and
                               direct launches                                  */
  int32_t refine;           /* refinement steps of the FP32 local solves (0: 1)  */
  int32_t tc_update;        /* FP32 factorizations: 1 trailing updates of fronts
                               beyond 96 rows on the tensor cores (tcgen05, operands
                               split into three TF32 parts, FP32 accumulation in
                               tensor memory); 0 or -1 (default): FP32 FMA units,
                               which are faster and more accurate in this release */
  int32_t reserved[7];
} bddc_options;

/* BDDC setup (Sec. 4-6) for the partition elem_to_subdomain (host [nE],
 * ids 0..N-1, each subdomain face-connected): interface classification into
 * macro vertices/edges/faces, primal constraints as an orthogonal change of
 * basis, nested-dissection multifrontal LDL^T factorizations of the
 * subdomain Dirichlet problems (Eq. uipi) and constrained Neumann problems
 * (zero-mean interior pressure, primal values fixed), the deluxe face
 * blocks (Sec. 6; with BDDC_SCALING_DELUXE_EDGES also the deluxe edge
 * blocks) and the coarse saddle matrix bordered by
 * sum_i |Omega_i| p_0,i = 0.  scaling: one of the BDDC_SCALING_* values,
 * else VEM_EINVAL.  opts may be NULL.  The handle keeps a pointer to sys,
 * which must outlive it.  Synchronizes. */
int bddc_setup(vem_system* sys, const int32_t* elem_to_subdomain, uint32_t constraints, int scaling,
               const bddc_options* opts, bddc** out);

/* z = M^{-1} r (Eq. BDDCprec) followed by the subdomain Dirichlet
 * (harmonic) extension; r, z: device system vectors (z overwritten).  The
 * interior velocity rows and the interior (zero-mean) pressure part of r
 * are ignored; only r on the interface DOFs and its subdomain-constant
 * pressure part enter, as in the interface problem (Eq. globInt). */
int bddc_apply(bddc* b, const double* r_dev, double* z_dev);

/* PCG on K u = f with the BDDC preconditioner; u0 = interior Dirichlet
 * solves so that every iterate is discrete-harmonic and the iteration is CG
 * on the interface problem (Eq. globInt).  Stops when the interface residual
 * (u_Gamma, p_0 parts) satisfies ||r||_2 <= rtol ||r_0||_2.  iters, kappa,
 * lam_min, lam_max (nullable): iteration count and the Lanczos estimates
 * from the CG coefficients.  f, u: device system vectors.  Returns
 * VEM_ENOTCONV at maxit, VEM_EBREAKDOWN if p^T K p <= 0.  Synchronizes. */
int pcg_solve(bddc* b, const double* f_dev, double* u_dev, double rtol, int maxit, int* iters, double* kappa,
              double* lam_min, double* lam_max);

/* Statistics by name: "n_subdomains", "n_coarse", "n_macro",
 * "factor_bytes_dirichlet", "factor_bytes_neumann", "n_deluxe_faces",
 * "n_deluxe_edges", "n_adaptive" (primal functionals added by the adaptive
 * coarse space), "t_adaptive_eig_ms", "deluxe_bytes", "deluxe_edge_bytes", "phi_bytes", "coarse_bytes", "n_front_max", and the setup
 * phase wall times "t_symbolic_ms", "t_upload_ms", "t_factor_dirichlet_ms",
 * "t_factor_neumann_ms", "t_factor_deluxe_ms", "t_deluxe_extract_ms",
 * "t_deluxe_combine_ms", "t_coarse_rhs_ms", "t_coarse_solves_ms",
 * "t_coarse_gram_ms", "t_coarse_inverse_ms"; "gib_free_after_<phase>" (free
 * device memory after each of those phases, GiB); "gflop_factor_dirichlet",
 * "gflop_factor_neumann", "gflop_factor_deluxe"; with the adaptive coarse
 * space the first setup's phases are kept as "first_<key>".  With the
 * environment variable VEMBDDC_SETUP_LOG set, each phase is also printed to
 * stderr as it ends. */
int bddc_info(bddc* b, const char* key, double* value);

/* Diagnostics: nrep forward+backward sweeps through all local Neumann and
 * Dirichlet factors (the triangular-solve part of one bddc_apply), timed
 * with CUDA events on the handle's stream.  *ms: average time of one
 * Neumann+Dirichlet sweep pair; *bytes: the factor bytes such a pair reads
 * (every panel once forward, once backward).  Synchronizes. */
int bddc_time_local_solves(bddc* b, int nrep, double* ms, double* bytes);
/* Diagnostics: one 128 x 128 x 32 tile product of the tensor-core front
 * update (tcgen05, three-part TF32 operand split, FP32 accumulation in
 * tensor memory, Sec. 4 local factorizations in FP32) on deterministic
 * data in [-1, 1), against an FP64 product.  *max_err: max |D - D_fp64|;
 * *max_ref: max |D_fp64|.  Returns VEM_ETIMEOUT if the bounded wait for the
 * product gave up.  Uses the current device; synchronizes it. */
int vem_tc_selftest(double* max_err, double* max_ref);
/* Diagnostics of failure detection: the bounded mbarrier wait that every
 * tensor-core kernel uses, run on an mbarrier that nothing ever arrives on,
 * polled at most `limit` times (0 <= limit <= 2^30).  Returns VEM_ETIMEOUT,
 * the status the tensor-core kernels report when their wait gives up, and
 * leaves the context usable; VEM_ECUDA if the wait completed; VEM_EINVAL
 * for a limit out of range.  No counterpart in the paper (failure
 * detection).  Uses the current device; synchronizes it. */
int vem_wait_selftest(long long limit);

int bddc_set_stream(bddc* b, void* cuda_stream);
void bddc_free(bddc* b);

#ifdef __cplusplus
}
#endif
#endif
