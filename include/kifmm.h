/*
 * kifmm.h -- C ABI of the GB300 kernel-independent fast multipole library for the
 * Laplace boundary sums of magnetostatic FEM-BEM and dielectric-polarization BEM
 * solvers (Jiang et al., "An O(N) and parallel approach to integral problems by a
 * kernel-independent fast multipole method").
 *
 * What is computed (raw sums, no 1/(4 pi)):
 *   f_i = sum_j K(r_i, r_j) q_j                                    Sec. II.A, Eq. sum_fmm
 *   KIFMM_KERNEL_SL  : K = 1/|r_i - r_j|                             the 1/r kernel (Sec. III.A.1)
 *   KIFMM_KERNEL_DL  : K = n_j.(r_i - r_j)/|r_i - r_j|^3             Eq. kernel (source normal)
 *   KIFMM_KERNEL_ADL : K = n_i.(r_i - r_j)/|r_i - r_j|^3             Eq. kernel_pol . n_i (Eq. Ax)
 *   KIFMM_KERNEL_FIELD: K = (r_i - r_j)/|r_i - r_j|^3, three outputs   Eq. kernel_pol (Eq. Eb, the
 *                      per target (x, y, z components, each an         field vector the force
 *                      n_trg block of the output)                      integrand needs)
 * with q_j = sigma_j w_j (density times quadrature weight) and the pair skipped
 * when |r_i - r_j| < 1e-5 (the tolerance radius of Sec. III.A.1).
 *
 * Conventions shared by every entry point:
 *  - Device pointers are CUDA device memory of the current device, owned by the
 *    caller, never retained after the call returns (geometry is copied into the
 *    tree / plan).  Host pointers are marked "host".
 *  - Coordinates and normals are structure-of-arrays of length 3n: x[0..n), then
 *    y[0..n), then z[0..n), FP64.
 *  - Outputs are in the caller's (input) point order.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream).
 *    Set-up calls and kifmm_bie_solve synchronize the stream before returning;
 *    kifmm_fmm_matvec, kifmm_quadrature_points and kifmm_polarization_rhs are
 *    asynchronous.
 *  - Every function returns KIFMM_OK (0) or a negative status; no exception
 *    crosses the ABI.  kifmm_last_error() returns a thread-local message for the
 *    last failure on the calling thread.
 *  - Handles are not thread-safe: one thread (and one stream) at a time per handle.
 */
#ifndef KIFMM_H
#define KIFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KIFMM_OK                 0
#define KIFMM_ERR_INVALID_ARG   (-1)  /* bad pointer, size, enum or handle            */
#define KIFMM_ERR_OOM           (-2)  /* device or host allocation failed               */
#define KIFMM_ERR_CUDA          (-3)  /* a CUDA call or kernel launch failed            */
#define KIFMM_ERR_NOT_CONVERGED (-4)  /* GMRES hit max_iter; x holds the last iterate   */
#define KIFMM_ERR_TIMEOUT       (-5)  /* a bounded device-side wait gave up             */
#define KIFMM_ERR_BREAKDOWN     (-6)  /* GMRES breakdown (zero or non-finite norm)      */
#define KIFMM_ERR_UNSUPPORTED   (-7)  /* a valid request this build does not implement  */

#define KIFMM_KERNEL_SL  0
#define KIFMM_KERNEL_DL  1
#define KIFMM_KERNEL_ADL 2
#define KIFMM_KERNEL_FIELD 3

#define KIFMM_PREC_FP64  0   /* every step in FP64 (the plain form)                        */
#define KIFMM_PREC_MIXED 1   /* FP32 near field and translations, FP64 set-up and output.
                                The double layers' near field forms n.(x - y) from hi + lo
                                splits whose hi products are exact in FP32, so that close
                                neighbours on curved surfaces lose nothing to cancellation. */

/* OR'ed into the precision argument of kifmm_fmm_setup: the far field by Chebyshev
   interpolation (the black-box FMM of the paper's ScalFMM: Sec. I and Sec. III.A.1, Eq.
   p2m) instead of equivalent densities, with p Chebyshev nodes per dimension in every
   box (Q = p^3, p in [2, 8]).  FP64 only.  The near field, the tree, the lists and the
   matvec's other steps are the same.                                                   */
#define KIFMM_ENGINE_CHEB 16

typedef struct kifmm_tree_s* kifmm_tree;
typedef struct kifmm_plan_s* kifmm_plan;
typedef struct kifmm_solver_s* kifmm_solver;

/* Last error message of the calling thread ("" if none).  Owned by the library. */
const char* kifmm_last_error(void);

/* Library version string, e.g. "kifmm 0.1 sm_103a". */
const char* kifmm_version(void);

/*
 * One-point quadrature on a triangle soup (Sec. III, electrostatic implementation):
 * the point is the triangle centroid; the weight is the spherical-triangle area
 * R^2 E (E the spherical excess) when the triangle lies on a sphere, else the flat
 * area; the normal is radial, (c - C)/|c - C|, on a sphere, else the unit facet
 * normal from the vertex winding.
 *   tri  device, n_tri*9 FP64: per triangle the 3 vertices (x,y,z) in order.
 *   sph  device, n_tri*4 FP64: sphere centre (x,y,z) and radius; radius <= 0 = flat.
 *   xyz, nrm  device, 3*n_tri FP64 SoA (outputs);  w  device, n_tri FP64 (output).
 * Errors: INVALID_ARG for NULL pointers or n_tri < 0; CUDA on a launch failure.
 */
int kifmm_quadrature_points(const double* tri, const double* sph, int64_t n_tri,
                            double* xyz, double* w, double* nrm, void* stream);

/*
 * Adaptive octree over sources (and targets) -- the target-source model of
 * Sec. III.A.1, with the octree depth set by a leaf capacity (the octree-height
 * knob of Sec. III.A.1 and IV.A).  Points are sorted by 63-bit Morton key (21 bits
 * per axis) in the smallest cube enclosing all points (enlarged by 1e-6 relative);
 * a box with more than max_leaf sources or targets is split, to depth <= 20.
 * Interaction lists U, V, W, X (Ying, Biros & Zorin 2004) are built on the device.
 *   src_xyz  device, 3*n_src FP64 SoA.      n_src >= 1.
 *   trg_xyz  device, 3*n_trg FP64 SoA, or NULL: targets are the sources.
 *   max_leaf 1..1024.
 *   out      host, receives the handle (NULL on failure).
 * Errors: INVALID_ARG (sizes, NULL, non-finite coordinates), OOM, CUDA.
 */
int kifmm_tree_build(const double* src_xyz, int64_t n_src,
                     const double* trg_xyz, int64_t n_trg,
                     int max_leaf, void* stream, kifmm_tree* out);

/*
 * Forest of independent instances in one tree (no counterpart in the paper, which
 * evaluates one boundary at a time): instance i is input points
 * [inst_off[i], inst_off[i+1]) and is both the sources and the targets of its own sum;
 * no instance sees another.  Each instance is translated (never scaled, so the sums,
 * the 1e-5 exclusion radius and the accuracy are those of the instance alone) into its
 * own cell of a 2^L x 2^L x 2^L grid, 8^L >= n_inst, with cells as wide as the widest
 * instance plus 1 %; the grid cells are the boxes of level L and no interaction list
 * crosses them.  Plans, matvecs and solves on the returned tree then run every FMM
 * phase as one launch for all instances, with inputs and outputs in the
 * concatenated input order.
 *   xyz       device, 3*n FP64 SoA, instances back to back.   1 <= n < 2^31.
 *   inst_off  host, n_inst+1 int64: 0 = inst_off[0] < inst_off[1] < ... = n.
 *   n_inst    1..KIFMM_MAX_INSTANCES.
 *   max_leaf, stream, out  as for kifmm_tree_build.
 * Errors: INVALID_ARG (sizes, offsets, empty instance, non-finite coordinates), OOM,
 * CUDA.
 */
#define KIFMM_MAX_INSTANCES 32768
int kifmm_forest_build(const double* xyz, int64_t n, const int64_t* inst_off, int n_inst,
                       int max_leaf, void* stream, kifmm_tree* out);

typedef struct {
    int64_t n_src, n_trg;
    int32_t n_boxes, n_leaves, n_levels, max_leaf;
    int64_t n_u, n_v, n_w, n_x;       /* total interaction-list entries           */
    int64_t p2p_pairs;                /* sum over target leaves of n_trg * U/W sources */
    double  root_center[3], root_half;
    int32_t n_instances;              /* 1, or the forest's instance count          */
    int32_t forest_level;             /* -1, or the level whose boxes are instances */
} kifmm_tree_stats;

/* Fill *stats (host).  Errors: INVALID_ARG. */
int kifmm_tree_get_stats(kifmm_tree tree, kifmm_tree_stats* stats);

/*
 * Copy the tree to host arrays (for inspection and tests).  Any pointer may be NULL.
 *   box_level[n_boxes], box_coord[3*n_boxes] (integer cell coordinates at the box's
 *   level, x y z per box), box_parent[n_boxes] (-1 for the root), box_leaf[n_boxes]
 *   (1 = leaf), box_range[4*n_boxes] (source begin, source end, target begin, target
 *   end in sorted order), src_perm[n_src], trg_perm[n_trg] (sorted position -> input
 *   index).  Boxes are ordered by level, then by Morton key.
 */
int kifmm_tree_export(kifmm_tree tree, int32_t* box_level, int32_t* box_coord,
                      int32_t* box_parent, int32_t* box_leaf, int64_t* box_range,
                      int64_t* src_perm, int64_t* trg_perm);

#define KIFMM_LIST_U 0
#define KIFMM_LIST_V 1
#define KIFMM_LIST_W 2
#define KIFMM_LIST_X 3
/*
 * Copy one interaction list in CSR form: offsets (host, n_boxes+1) and idx (host,
 * offsets[n_boxes] entries, source box ids).  Either pointer may be NULL; call with
 * idx == NULL first to size it from offsets[n_boxes].
 */
int kifmm_tree_export_list(kifmm_tree tree, int which, int64_t* offsets, int32_t* idx);

/* Release a tree.  Plans built on it must be destroyed first.  NULL is a no-op. */
int kifmm_tree_destroy(kifmm_tree tree);

/*
 * Plan: translation operators and per-leaf evaluation matrices for one kernel,
 * order and precision on a tree.  KIFMM operators (Ying, Biros & Zorin 2004) with
 * surfaces of p points per cube edge (Q = 6(p-1)^2 + 2 points), equivalent surfaces
 * at 1.05 and check surfaces at 2.95 box half-widths; the check-to-equivalent
 * pseudo-inverses come from an FP64 SVD truncated at pinv_cutoff * sigma_max and are
 * folded into every operator, so the matvec only moves check potentials.
 * The double-layer normal is applied at the source-to-check step (Sec. III.A.1,
 * Eq. p2m, the "second method"); the adjoint target normal at evaluation.
 *   kernel      KIFMM_KERNEL_SL / DL / ADL / FIELD.
 *   p           2..16.
 *   precision   KIFMM_PREC_FP64 or KIFMM_PREC_MIXED; KIFMM_PREC_FP64 | KIFMM_ENGINE_CHEB
 *               selects the Chebyshev-interpolation far field (p: nodes per dimension).
 *   pinv_cutoff > 0 and < 1: both pseudo-inverses truncated there; or 0 for the
 *               defaults: FP64 1e-9; mixed 1e-8, except Pu of the double layer at 1e-9
 *               (the dipole sources' upward densities need those directions).  The
 *               mixed form also keeps at most 256 singular triplets of Pd, and of Pu
 *               except for the double layer (from p = 11 on, 1e-8 would keep more):
 *               the rows one tensor-core work item covers.  The ranks kept are in
 *               kifmm_plan_get_stats (rank_up, rank_down).
 *   src_nrm     device 3*n_src SoA; required for DL, else ignored (may be NULL).
 *   trg_nrm     device 3*n_trg SoA; required for ADL, else ignored (may be NULL).
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int kifmm_fmm_setup(kifmm_tree tree, int kernel, int p, int precision, double pinv_cutoff,
                    const double* src_nrm, const double* trg_nrm,
                    void* stream, kifmm_plan* out);

/*
 * f = K q for all targets (see the top of this file).
 *   q    device, n_src FP64 (density times weight), input order.
 *   out  device, n_trg FP64, input order (overwritten); KIFMM_KERNEL_FIELD: 3 n_trg,
 *        the x components of all targets, then y, then z.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA.
 */
int kifmm_fmm_matvec(kifmm_plan plan, const double* q, double* out, void* stream);

/*
 * The same matvec replayed from a CUDA graph (no counterpart in the paper): the
 * first call for a given (q, out) pair captures one matvec's launches on a private
 * stream and instantiates them; every call then launches the graph on `stream`, so
 * a matvec costs one launch on the host whatever the tree's depth.  The graph reads
 * q and writes out by address: refill q in place between calls.  A call with other
 * pointers captures again.  Profiling events are not recorded inside the graph.
 * Errors: INVALID_ARG, CUDA (capture or instantiation failed; the plan stays usable
 * through kifmm_fmm_matvec).
 */
int kifmm_fmm_matvec_graph(kifmm_plan plan, const double* q, double* out, void* stream);

/*
 * The matvec with q and out in host memory (no counterpart in the paper; for callers
 * whose densities live on the host).
 *   q      n_src FP64, input order.  Page-locked host memory (cudaHostAlloc,
 *          cudaHostRegister, a pinned torch tensor): the first kernel reads it in place,
 *          each element once and in order (on Grace systems over NVLink-C2C, with no
 *          separate copy).  Pageable host memory: copied to a device staging buffer by
 *          cudaMemcpyAsync.  Device memory: read as kifmm_fmm_matvec reads it.
 *   out    n_trg FP64, input order, overwritten.  Page-locked: the last kernel writes
 *          it in place, each element once and in order.  Pageable: copied back from
 *          a device staging buffer after the matvec.  Device: written as by
 *          kifmm_fmm_matvec.
 *   graph  0: launch the kernels; 1: replay a graph captured for this (q, out) pair,
 *          as kifmm_fmm_matvec_graph does (captured again when the pair changes).
 * Asynchronous on `stream` for page-locked and device buffers: synchronize before
 * reading out or refilling q.  The first call allocates the inverse permutations and
 * the staging buffer of the near sums (8 bytes per source, 16 per target), the first
 * pageable q a staging buffer of 8 bytes per source.  The results are
 * kifmm_fmm_matvec's, up to the order of its atomic sums (which varies from run to run
 * in either).  Errors: INVALID_ARG, OOM, CUDA.
 */
int kifmm_fmm_matvec_host(kifmm_plan plan, const double* q, double* out, int graph, void* stream);

typedef struct {
    int32_t kernel, p, q_points, precision;
    double  pinv_cutoff;              /* truncation of the downward pseudo-inverse Pd   */
    int64_t device_bytes;             /* device memory held by the plan      */
    int64_t m2l_pairs, u2u_pairs, l2l_pairs, s2u_leaves, x_pairs;
    int32_t launches_per_matvec;      /* kernels one kifmm_fmm_matvec enqueues */
    int32_t rank_up, rank_down;       /* numerical ranks of the up / down check-to-
                                         equivalent pseudo-inverses at pinv_cutoff   */
    int32_t m2l_width;                /* columns of each M2L' operator as applied:
                                         q_points (FP64) or rank_up (mixed: M2L' acts
                                         on the projections onto Pu's range)          */
    int32_t m2l_rows;                 /* its rows: q_points (FP64) or rank_down (mixed:
                                         it yields the projection onto Pd's range)    */
    int32_t near_units;               /* mixed: near-field work units (one pass of a
                                         target leaf's targets over at most 2048 of
                                         its sources)                                  */
    int32_t near_split_leaves;        /* mixed: target leaves spread over several
                                         units (their sums meet by FP64 atomics)      */
    int32_t near_overlap;             /* 1: the near field runs on its own (lowest-
                                         priority) stream beside the far field -- from
                                         the gather on, or after M2L when it evaluates
                                         fewer than 100 pairs per target -- so its
                                         profiled phase time spans the overlap         */
    int32_t s2u_points;               /* up-check points S2U evaluates: q_points (FP64)
                                         or the skeleton of kifmm_up_skeleton (mixed)  */
    int64_t m2l_chain_pairs;          /* mixed: V pairs in M2L chains -- runs of at most
                                         128 targets of one level whose V lists hold the
                                         same offsets, whose products over all of those
                                         offsets are summed on chip and written once    */
    double  pinv_cutoff_up;           /* truncation of the upward pseudo-inverse Pu     */
    int64_t near_corr_ranges;         /* mixed: near-field source ranges with a pair closer
                                         than 1/32 of the range's extent or within 4x the
                                         tolerance radius, evaluated with the distance
                                         corrected for the FP32 offsets' rounding         */
    int64_t near_pairs;               /* (target, source) pairs of the near field (U, W
                                         and leaf X lists) per matvec                    */
    int32_t near_axis_units;          /* mixed DL: near-field units whose source normals
                                         all lie along one coordinate axis (flat faces
                                         normal to an axis), evaluated with the one-term
                                         n.(x - y) of those normals                      */
    double  setup_ms[5];              /* wall-clock set-up time (ms), device work included:
                                         [0] operator tables (0 when shared with a live
                                         plan of the same key), [1] work lists and the
                                         near-field units, [2] translation tiles, [3]
                                         evaluation rows, [4] the total                    */
    int64_t near_axis_pairs;          /* mixed DL: the pairs of those axis units         */
    int64_t near_zero_pairs;          /* DL: pairs left out because they add exactly
                                         zero -- a source box whose dipoles all lie along
                                         one coordinate axis and whose points all share
                                         the target leaf's coordinate along it
                                         (n.(x - y) = 0); not in near_pairs            */
} kifmm_plan_stats;

int kifmm_plan_get_stats(kifmm_plan plan, kifmm_plan_stats* stats);

/*
 * Skeleton of the upward check surface of order p (host only: no device work).  The
 * paper's S2U (Sec. III.A.2, the source-to-up-check step of the upward pass) evaluates
 * the sources' potential at all Q = 6(p-1)^2 + 2 check points; the mixed form evaluates
 * it at k of them and interpolates the rest, an interpolative decomposition that is
 * not in the paper.  The k points are the first k pivots of a column-pivoted
 * Householder QR of K(e_j, c_i) (rows: the Q upward equivalent points at 1.05
 * half-widths, columns: the Q check points at 2.95), in FP64.  Then the potential of
 * any source inside the box satisfies u(c_i) = sum_m E[i][m] u(c_idx[m]) up to that
 * QR's truncation.
 *   p      expansion order, 2..16.
 *   k      skeleton size, 1..Q.
 *   idx    host, k int32 or NULL: check-point indices of the skeleton.  Points are
 *          numbered as kifmm's unit surface: the boundary points of the p x p x p grid
 *          on [-1, 1]^3, x outermost, then y, then z.
 *   E      host, Q x k doubles (row-major) or NULL: the interpolation matrix.
 *   k_tol  host, 1 int32 or NULL: pivots with |R_ii| > 1e-9 |R_00| (how many a
 *          mixed plan starts from before rounding up to its surface kernel's shape).
 * Errors: INVALID_ARG (p or k out of range).
 */
int kifmm_up_skeleton(int p, int k, int32_t* idx, double* E, int32_t* k_tol);

/*
 * Per-phase device times (milliseconds).  While enabled, every matvec records CUDA
 * events between its phases on its stream (no host synchronization).  A call with
 * phases != NULL (host, >= 9 doubles) waits for the recorded events and returns the
 * mean per matvec since the previous read: {gather, s2u, u2u, x, m2l, l2l, d2t, p2p,
 * total}; then recording is switched on (enable != 0) or off.  enable = 2 also runs
 * the near field after the far field on the matvec's stream instead of beside it, so
 * that p2p is the near field's own time with the whole GPU (a roofline measurement;
 * the results do not change); enable = 1 keeps the overlapped schedule, in which p2p
 * spans the far field it runs beside.
 */
int kifmm_plan_profile(kifmm_plan plan, int enable, double* phases);

/*
 * Health check of the plan's device work (synchronizes with the device).  The
 * tensor-core translation GEMMs bound every pipeline wait; a wait that gives up
 * records a code in a device word of the plan, skips its writes and frees its
 * tensor memory.  Returns KIFMM_ERR_TIMEOUT if that ever happened, else KIFMM_OK.
 */
int kifmm_plan_check(kifmm_plan plan);

/* Release a plan.  NULL is a no-op. */
int kifmm_plan_destroy(kifmm_plan plan);

/*
 * Right-hand side of the polarization system for a uniform applied field and no
 * free charge: b_j = -(eps_out - eps_j) E0 . n_j   (Eq. rhs with sigma_f = 0 and the
 * free-charge field replaced by E0).
 *   nrm device 3n SoA, eps_in device n, b device n (output).
 */
int kifmm_polarization_rhs(const double* nrm, const double* eps_in, double eps_out,
                           const double e0[3], int64_t n, double* b, void* stream);

/*
 * Solve the dielectric polarization system A sigma = b (Sec. II.C, Eqs. Ax, Eb,
 * pol_discret) matrix-free with restarted GMRES(restart) in FP64 (Sec. III), on a
 * plan built with KIFMM_KERNEL_ADL on targets = sources:
 *   (A s)_j = ebar_j s_j + deps_j (1/4pi) [ ADL(s * area)_j + c_j s_j ],
 *   ebar_j = (eps_j + eps_out)/2,  deps_j = eps_out - eps_j,  c_j = H_j sqrt(pi a_j)
 * (the self-patch correction: principal-value normal field of a disc of area a_j
 * on a surface of mean curvature H_j).  Krylov basis, orthogonalization (classical
 * Gram-Schmidt applied twice) and residuals are FP64 on the device; x0 is the
 * content of x on entry.  Stops when the GMRES residual estimate falls to
 * tol * ||b|| and returns the true relative residual ||b - A x||/||b|| in *rel_res.
 * On a forest (kifmm_forest_build) every instance is solved by its own GMRES -- its
 * own Krylov coefficients, residual and stopping test on its segment of the vectors --
 * and all instances share each step's matvec (one launch per phase for all of
 * them); an instance that has stopped takes zero basis vectors until the others
 * stop.  *iters is then the number of shared steps and *rel_res the largest
 * instance's true residual; kifmm_solver_instances gives them per instance.
 *   area, eps_in, curv, b: device, n FP64 (input order);  x device n (in/out).
 *   iters, rel_res: host (may be NULL).
 * Errors: INVALID_ARG, OOM, CUDA, NOT_CONVERGED (x = last iterate), BREAKDOWN (on a
 * forest: the first failing instance's status).
 */
int kifmm_bie_solve(kifmm_plan plan, const double* area, const double* eps_in, double eps_out,
                    const double* curv, const double* b, double* x,
                    double tol, int restart, int max_iter,
                    int* iters, double* rel_res, void* stream);

/*
 * The same GMRES as kifmm_bie_solve, advanced one step at a time so that several
 * solves can share the GPU (no counterpart in the paper, which solves one system at a
 * time).  A step is one of: the norm of b, a restart (one matvec), one Arnoldi
 * iteration (one matvec and two Gram-Schmidt passes), the final true residual (one
 * matvec).
 *   kifmm_solver_create: arguments as kifmm_bie_solve; area, eps_in, curv, b and x
 *     must stay allocated until the solver is destroyed (x is updated in place).  The
 *     solver owns its Krylov basis ((restart+1) n FP64), so several solvers may share
 *     one plan -- but their steps must then not overlap on the GPU (the plan's
 *     matvec buffers are shared): launch and finish them one after the other.
 *   kifmm_solver_launch: enqueue the next step's device work on `stream`; returns
 *     without waiting.
 *   kifmm_solver_finish: wait for that work and advance on the host.  *done = 1 once
 *     the solve has ended; *iters = Arnoldi iterations so far; *rel_res = the GMRES
 *     residual estimate, or after the end the true relative residual.  Returns the
 *     solve's status once it has ended (OK, NOT_CONVERGED, BREAKDOWN), else OK.
 * Launch and finish alternate; solvers on different plans and streams may each be
 * launched before any is finished, which overlaps their device work.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int kifmm_solver_create(kifmm_plan plan, const double* area, const double* eps_in, double eps_out,
                        const double* curv, const double* b, double* x, double tol, int restart,
                        int max_iter, kifmm_solver* out);
int kifmm_solver_launch(kifmm_solver solver, void* stream);
int kifmm_solver_finish(kifmm_solver solver, int* done, int* iters, double* rel_res);
int kifmm_solver_destroy(kifmm_solver solver);

/*
 * Per-instance state of a solver on a forest (on one tree: n_inst = 1).
 *   n_inst  the tree's instance count (kifmm_tree_get_stats n_instances).
 *   iters   host, n_inst: the shared step at which each instance last advanced.
 *   rel_res host, n_inst: the GMRES residual estimate, or after the end the true
 *           relative residual ||b_i - A_i x_i|| / ||b_i||.
 *   status  host, n_inst: OK while running; after the end OK, NOT_CONVERGED or BREAKDOWN.
 * Any array may be NULL.  Errors: INVALID_ARG (NULL solver, n_inst mismatch).
 */
int kifmm_solver_instances(kifmm_solver solver, int n_inst, int32_t* iters, double* rel_res,
                           int32_t* status);

/*
 * The polarization operator itself, y = A x (same definition as kifmm_bie_solve).
 * Asynchronous.
 */
int kifmm_bie_apply(kifmm_plan plan, const double* area, const double* eps_in, double eps_out,
                    const double* curv, const double* x, double* y, void* stream);

/*
 * Right-hand side of the polarization system with free surface charge (Eq. rhs, with
 * Eq. Ef without its volume term -- no free charge in the medium):
 *   b_j = (1 - ebar_j) sf_j - deps_j [ E0 . n_j + (1/4pi) ( ADL(sf * a)_j + c_j sf_j ) ]
 * the free charge's own field at the elements discretized as Eq. pol_discret (with the
 * self-patch term of kifmm_bie_solve), on a plan built with KIFMM_KERNEL_ADL on
 * targets = sources.  With sf = 0 this is kifmm_polarization_rhs.
 *   area, eps_in, curv, sigma_f, b (output): device, n FP64;  nrm device 3n SoA;
 *   e0 host, 3 doubles.  Asynchronous.  Errors: INVALID_ARG, OOM, CUDA.
 */
int kifmm_polarization_rhs_free(kifmm_plan plan, const double* area, const double* eps_in, double eps_out,
                                const double* curv, const double* nrm, const double* sigma_f,
                                const double e0[3], double* b, void* stream);

/*
 * Electrostatic field at the surface elements (Sec. II.C, Eq. Eb discretized as Eq.
 * pol_discret, with the applied uniform field E0):
 *   E^j = E0 + (1/4pi) [ sum_{k != j} (r_j - r_k)/|r_j - r_k|^3 sigma_k a_k + c_j sigma_j n_j ]
 * c_j = H_j sqrt(pi a_j) as in kifmm_bie_solve; sigma is the total surface charge
 * (free plus bound).  On a plan built with KIFMM_KERNEL_FIELD on targets = sources.
 *   area, curv, sigma: device, n FP64;  nrm device 3n SoA;  e0 host, 3 doubles;
 *   E: device, 3n FP64 (output, x of all elements, then y, then z).
 * Asynchronous.  Errors: INVALID_ARG, OOM, CUDA.
 */
int kifmm_polarization_field(kifmm_plan plan, const double* area, const double* curv, const double* nrm,
                             const double* sigma, const double e0[3], double* E, void* stream);

/*
 * Electrostatic force on each body (Sec. II.C: F_i = integral over body i of the surface
 * force density f = eps_m sigma E), with the one-point rule:
 *   F_b = sum over the elements j of body b of eps_out sigma_j E^j a_j
 * and E^j of kifmm_polarization_field (same plan and arguments).
 *   body: device, n int32, the body of each element (elements outside [0, n_body) are
 *         skipped);  n_body >= 1.
 *   F: device, 3 n_body FP64 (output): F[3 b + k] is component k of body b's force.
 * Asynchronous; uses 3n doubles of the plan's scratch.  The per-body sums meet by FP64
 * atomics, so their rounding order varies from run to run.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int kifmm_polarization_force(kifmm_plan plan, const double* area, const double* curv, const double* nrm,
                             const double* sigma, double eps_out, const double e0[3], const int32_t* body,
                             int n_body, double* F, void* stream);

/*
 * Demagnetizing-field boundary potential of the Fredkin-Koehler split (Sec. II.B,
 * Eq. fk_integral_discrete):
 *   phi2_i = (1/4pi) sum_j n_j.(r_i - r_j)/|r_i - r_j|^3 phi1_j w_j + (Omega_i/4pi - 1) phi1_i
 * on a plan built with KIFMM_KERNEL_DL on targets = sources.
 *   phi1, w, omega (solid angle), phi2 (output): device, n FP64.  Asynchronous.
 */
int kifmm_demag_phi2(kifmm_plan plan, const double* phi1, const double* w,
                     const double* omega, double* phi2, void* stream);

/*
 * kifmm_demag_phi2 without any device allocation (the paper has no counterpart; this
 * is a library-level convenience).  For callers that cannot allocate device memory
 * when they evaluate phi2: a pooled or custom allocator that forbids driver
 * allocations, a loop that cannot afford cudaMalloc's implicit synchronization, or
 * work being recorded into a CUDA graph.  Same arguments and result as
 * kifmm_demag_phi2; the scratch vector phi1 * w is kept in a static device array of
 * 2^20 doubles (8 MiB) that every device holds while the library is loaded.
 *  - Plans with more than 2^20 targets are rejected with KIFMM_ERR_INVALID_ARG.
 *  - The first call on a device looks up that array's device address (once per
 *    device); make that first call before any stream capture begins.  With lazy
 *    module loading (the CUDA default) that first call may also be what loads the
 *    library's module on the device, and so what reserves the array's 8 MiB (a driver
 *    allocation).  From the second call on, nothing is allocated.
 *  - All calls share the one array, so calls that can overlap on the GPU (different
 *    streams, or different plans without ordering between them) race on it.
 *  - No cudaMalloc, cudaFree or allocating library routine is called.  Asynchronous.
 */
int kifmm_demag_phi2_noalloc(kifmm_plan plan, const double* phi1, const double* w,
                             const double* omega, double* phi2, void* stream);

/*
 * Peak-rate microbenchmark (no counterpart in the paper: it measures the
 * denominators of the roofline fractions the library's kernels are reported
 * against).  One kernel per unit issues only that arithmetic instruction, on eight
 * independent chains per thread, from every resident thread of every SM of the
 * current device; the launch is sized to about 10 ms and timed with CUDA events on
 * `stream`, `reps` times.
 *   unit  KIFMM_PEAK_FP32_FMA (fmaf), KIFMM_PEAK_FP32X2_FMA (packed __ffma2_rn),
 *         KIFMM_PEAK_RSQRT (rsqrtf, the near field's reciprocal square root),
 *         KIFMM_PEAK_FP64_FMA (fma on doubles).
 *   rate  host, receives the best rate: flops/s for the FMA units (an FMA counts 2,
 *         a packed FMA 4), reciprocal square roots/s for KIFMM_PEAK_RSQRT.
 *   ms    host or NULL, receives the best launch time.
 * Synchronizes `stream`.  Allocates 2 KB of device memory for the kernels' sink.
 * Errors: INVALID_ARG (unit outside 0..3, reps outside 1..100), OOM, CUDA.
 */
#define KIFMM_PEAK_FP32_FMA   0
#define KIFMM_PEAK_FP32X2_FMA 1
#define KIFMM_PEAK_RSQRT      2
#define KIFMM_PEAK_FP64_FMA   3
int kifmm_peak_rate(int unit, int reps, double* rate, double* ms, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* KIFMM_H */
