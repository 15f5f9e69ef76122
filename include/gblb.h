/* gblb.h -- C ABI of the GB300 Laplace-Beltrami layer-potential library.
 *
 * The library discretises closed surfaces made of curved triangular patches
 * (Section 4 of Agarwal, O'Neil & Rachh, "FMM-accelerated solvers for the
 * Laplace-Beltrami problem on complex surfaces in three dimensions") and
 * applies, on one CUDA device, the layer potentials S, D, S', S''+D' and
 * grad S (Section 3), the second-kind operators A2 and A3 (Sections 4.2 and
 * 4.3), and solves the mean-zero Laplace-Beltrami problem
 * Delta_Gamma u = f (Section 2, Lemma 1) with GMRES (Section 6).  The Hodge
 * decomposition of a tangential field into curl-free, divergence-free and
 * harmonic parts (Section 5) is built on the solver.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: LB_OK (0) or a negative LB_E*
 *     code.  A human-readable message for the last failure on a context is
 *     returned by lb_last_error().  No C++ exception crosses this boundary.
 *   - N = npatch * np nodes, patch-major: node index = patch * np + q, where
 *     q indexes the reference nodes on T0 = {u, v >= 0, u + v <= 1}.
 *   - Vectors over nodes are float64, contiguous.  A batch of nrhs vectors is
 *     stored [nrhs][N].  Vector fields are [N][3] (or [nrhs][N][3]).
 *   - Pointers marked "host or device" may point to host memory (pageable or
 *     pinned) or to device memory of the context's device; the library looks
 *     up the pointer kind and copies host data through its own device
 *     buffers.  Pointers marked "device" must be device memory.
 *   - All device work is enqueued on the context's stream (lb_set_stream);
 *     entry points that return host-visible results (solve information,
 *     host output buffers) synchronise that stream before returning.
 *   - The caller keeps ownership of every pointer it passes; the library
 *     copies what it needs.  The context owns all device memory it allocates
 *     and frees it in lb_destroy().
 *   - Contexts are not thread-safe: use one context per host thread.
 */
#ifndef GBLB_H
#define GBLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LB_OK 0
#define LB_EINVAL (-1)         /* bad argument (null pointer, size, non-finite input) */
#define LB_ENOMEM (-2)         /* device or host allocation failed */
#define LB_ECUDA (-3)          /* a CUDA runtime call failed */
#define LB_ENOTCONVERGED (-4)  /* GMRES hit max_iter before tol; best iterate written */
#define LB_ETIMEOUT (-5)       /* a bounded device-side wait expired */
#define LB_EGEOM (-6)          /* degenerate geometry (zero Jacobian, bad node rule) */
#define LB_ESTATE (-7)         /* call out of order (e.g. apply before geometry) */

/* arithmetic of the far-field pair sums (the rest of the path is float64) */
#define LB_FP64 0          /* float64 pairs */
#define LB_FP32 1          /* float32 pairs, compensated accumulation */
#define LB_FP32_REFINED 2  /* solve: float32 inner GMRES inside refinement whose residual and
                              solution potentials use LB_DF64 pair sums */
#define LB_DF64 3          /* double-float pairs: every quantity as a float32 pair hi + lo,
                              error-free transformations, about 1e-14 relative */

/* integral-equation formulation (Section 4, Table 2) */
#define LB_A1 1   /* u = S[sigma]:   div S grad_Gamma S [sigma] + SWS[sigma] = S[f] (Section 4.1,
                     eq. ie-dis0; not second kind: the comparison case of Section 6.2) */
#define LB_A2 2   /* u = S[sigma]:   -sigma/4 + D^2 - S(S''+D'+2HS') + SWS = S[f]  */
#define LB_A3 3   /* u = S^2[sigma]: -sigma/4 + S'^2 - (S''+D'+2HS')S + WS^2 = f    */

/* kernels of the near-field correction blocks, in storage order */
#define LB_K_S 0
#define LB_K_D 1
#define LB_K_SP 2
#define LB_K_SPPDP 3
#define LB_NKERNELS 4

typedef struct lb_ctx lb_ctx;   /* opaque */

typedef struct {
  double eps_quad;      /* near-field quadrature tolerance (Section 6: epsilon); default 1e-12 */
  double near_factor;   /* eta: patch P is near node x when |x - c_P| < eta * R_P; default 2 */
  int precision;        /* LB_FP64, LB_FP32, LB_FP32_REFINED or LB_DF64; default LB_FP64 */
  int formulation;      /* LB_A3, LB_A2 or LB_A1; default LB_A3 */
  int max_iter;         /* GMRES iteration cap (Section 6 caps at 100); default 100 */
  double tol;           /* relative residual target |b - A x| / |b|; default 1e-10 */
  double inner_tol;     /* LB_FP32_REFINED: inner GMRES relative tolerance; default 1e-5 */
  int max_refine;       /* LB_FP32_REFINED: outer refinement steps cap; default 6 */
  int graphs;           /* 1: lockstep solves replay each GMRES iteration as a captured CUDA graph
                           (while per-kernel profiling is off); 0: plain launches; default 1 */
} lb_params;

typedef struct {
  int32_t iterations;       /* total GMRES iterations (inner iterations when refined) */
  int32_t refinements;      /* outer refinement steps (0 for a plain solve) */
  int32_t converged;        /* 1 if every right-hand side reached tol */
  int32_t applies_fp64;     /* operator applies with float64 or double-float pair sums */
  int32_t applies_fp32;     /* operator applies with float32 pair sums */
  int32_t nrhs;
  double rel_residual;      /* worst final relative residual over the batch (float64 apply) */
  double removed_mean;      /* weighted mean removed from the first right-hand side */
  double history[128];      /* relative residual estimate per GMRES iteration, first rhs */
  int32_t history_len;
  int64_t pairs;            /* far-field pair interactions evaluated by the solve */
  int32_t graph_iterations; /* lockstep GMRES iterations run as CUDA-graph replays */
} lb_solve_info;

typedef struct {
  int64_t N;            /* number of nodes */
  int64_t npatch;
  int32_t np;           /* nodes per patch, (order+1)(order+2)/2 */
  int32_t order;        /* total degree of the patch polynomials */
  int64_t nnzb;         /* near (row, patch) blocks; 0 before near lists exist */
  double area;          /* sum of the smooth weights */
  int32_t sm_count;     /* multiprocessors of the device */
  int32_t corrections;  /* 1 when correction blocks are present */
} lb_geom_info;

/* Fill *p with the defaults listed above. */
int lb_default_params(lb_params* p);

/* Create a context on CUDA device `device` with parameters *p (NULL: defaults).
 * *out receives the context.  Errors: LB_EINVAL, LB_ECUDA, LB_ENOMEM. */
int lb_create(lb_ctx** out, int device, const lb_params* p);

/* Release every device buffer of the context and the context itself.
 * Accepts NULL. */
int lb_destroy(lb_ctx* ctx);

/* Message for the last failing call on ctx (static string when ctx is NULL). */
const char* lb_last_error(const lb_ctx* ctx);

/* Replace the solver parameters.  Changing eps_quad or near_factor drops the
 * near lists and corrections, which must then be rebuilt. */
int lb_set_params(lb_ctx* ctx, const lb_params* p);
int lb_get_params(const lb_ctx* ctx, lb_params* p);

/* Enqueue all later work on `stream` (a cudaStream_t, NULL = legacy default). */
int lb_set_stream(lb_ctx* ctx, void* stream);

/* Upload a surface (Section 4: charts X^j : T0 -> Gamma_j sampled at an
 * order-`order` node rule).
 *   ref_uv [np][2], ref_w [np]: reference nodes and smooth weights on T0
 *     (host or device); np must equal (order+1)(order+2)/2 and sum(ref_w)
 *     must be 1/2.
 *   X, Xu, Xv [N][3]: chart samples and their u/v derivatives (host or device),
 *     oriented so that Xu x Xv points outward.
 * Computes on the device (Sections 2 and 4): unit normals, weights
 * w = ref_w |Xu x Xv|, the inverse metric, the mean curvature
 * H = -1/2 tr(g^-1 L) from nodal differentiation of Xu and Xv, patch
 * centroids and radii.  Drops earlier near lists and corrections.
 * Errors: LB_EINVAL (sizes, node rule), LB_EGEOM (|Xu x Xv| = 0), LB_ENOMEM. */
int lb_upload_geometry(lb_ctx* ctx, int64_t npatch, int order, const double* ref_uv,
                       const double* ref_w, const double* X, const double* Xu,
                       const double* Xv);

/* Copy the derived node quantities to caller buffers (host or device; any may
 * be NULL): normals n [N][3], weights w [N], mean curvature H [N]. */
int lb_get_geometry(lb_ctx* ctx, double* n, double* w, double* H);

int lb_geometry_info(lb_ctx* ctx, lb_geom_info* info);

/* Build the near lists Near(i) = {P : |x_i - c_P| < eta R_P} (Section 4,
 * the Near/Far split) on the device. */
int lb_build_near(lb_ctx* ctx);

/* Build the near-field correction blocks (Section 4, the corrected weights
 * w~_ij composed with polynomial interpolation on each near patch): for
 * every row i and P in Near(i), W^K_{i,P}[q] = int_P K(x_i, y) l_q(y) da(y)
 * for K in {S, D, S', S''+D'}, by adaptive quadrature on the device (Duffy
 * maps on the self patch, 1-to-4 subdivision on the others) to eps_quad.
 * Builds the near lists first if needed.  This is the setup cost t_q of
 * Section 6, amortised over the solve. */
int lb_build_corrections(lb_ctx* ctx);

/* Load externally computed near lists and correction blocks instead of
 * building them (host or device pointers):
 *   row_ptr [N+1] (int64): blocks of row i are row_ptr[i] .. row_ptr[i+1]-1,
 *   patch [nnzb] (int32): the near patch of each block, ascending per row,
 *   vals [nnzb][4][np] (float64): the weights, kernel order S, D, S', S''+D'.
 * The far-field sums skip exactly these (row, patch) pairs.  The lists are
 * checked on the device before they are kept: row_ptr must run from 0 to
 * nnzb without decreasing, every patch index must lie in [0, npatch) and the
 * patches of a row must be strictly ascending; LB_EINVAL otherwise (nothing is
 * kept).  The library cannot check the size of a host vals buffer: it must
 * hold nnzb * 4 * np doubles. */
int lb_load_corrections(lb_ctx* ctx, int64_t nnzb, const int64_t* row_ptr,
                        const int32_t* patch, const double* vals);

/* Copy the current near lists / corrections out (host or device buffers of
 * the sizes above; vals may be NULL to fetch the lists only). */
int lb_get_corrections(lb_ctx* ctx, int64_t* row_ptr, int32_t* patch, double* vals);

/* Oversampled far-field rule (Section 4: the smooth far-field quadrature runs
 * on an oversampled rule; the paper gives no oversampling factor).  uv
 * [nps][2], w [nps] (host or device) are a node rule of total degree `order`
 * on T0 (nps = (order+1)(order+2)/2, nodes in T0, weights summing to 1/2).
 * On every patch the chart X, its tangents X_u, X_v and, in every later pass,
 * the density are interpolated from the node rule to these nodes (the
 * Lagrange polynomials of the node rule); the far sums then run over the
 * npatch * nps interpolated points with normals and area elements of the
 * interpolated tangents, weights w |X~_u x X~_v|.  Near corrections are
 * unchanged.  Applies to every single-density pass (lb_far_sums, the
 * potentials, lb_apply_A, the solves and harmonic fields, which then solve
 * their right-hand sides one by one); the transposed applies, the adjoint
 * solve and the node-position gradient return LB_EINVAL while a far rule is
 * set.  order 0 (uv, w ignored) restores the node rule.  Dropped by
 * lb_upload_geometry.  Errors: LB_ESTATE (no geometry), LB_EINVAL. */
int lb_set_far_rule(lb_ctx* ctx, int order, const double* uv, const double* w);

/* Far-field sums alone (Section 4: the target-independent smooth rule over
 * all sources outside Near(i)): out [nrhs][4][N] (host or device) receives
 * sum_{j far} w_j K(x_i, x_j) sigma_j for K = S, D, S', S''+D', computed with
 * `precision` (LB_FP64, LB_FP32 or LB_DF64).  sigma [nrhs][N] host or device. */
int lb_far_sums(lb_ctx* ctx, int precision, int nrhs, const double* sigma, double* out);

/* Discretised potentials, far sum + near corrections (Section 4):
 * out [nrhs][N] = K[sigma] for K = S, S', D, S''+D'.  sigma, out: host or
 * device.  Far pairs use the context's precision (FP32_REFINED -> FP32). */
int lb_apply_S(lb_ctx* ctx, int nrhs, const double* sigma, double* out);
int lb_apply_Sp(lb_ctx* ctx, int nrhs, const double* sigma, double* out);
int lb_apply_D(lb_ctx* ctx, int nrhs, const double* sigma, double* out);
int lb_apply_SppDp(lb_ctx* ctx, int nrhs, const double* sigma, double* out);

/* grad S on Gamma: out [nrhs][N][3] = n S'[sigma] + grad_Gamma S[sigma]
 * (the principal-value gradient: normal part S', tangential part the surface
 * gradient of the continuous potential S[sigma], by nodal differentiation
 * within each patch, Section 2). */
int lb_apply_gradS(lb_ctx* ctx, int nrhs, const double* sigma, double* out);

/* The operator of the context's formulation (A3 or A2; Sections 4.2, 4.3):
 * out [nrhs][N] = A tau.  tau, out: host or device.  With A3, nrhs >= 2 and
 * float32 or double-float pairs, up to 8 densities share each far-field
 * pass (the pair geometry is evaluated once for all of them). */
int lb_apply_A(lb_ctx* ctx, int nrhs, const double* tau, double* out);

/* Solve Delta_Gamma u = f for mean-zero u (Lemma 1), nrhs right-hand sides
 * at once: f is projected to weighted mean zero, GMRES (x0 = 0, no restart,
 * Euclidean norm, at most max_iter iterations) solves A sigma = b with
 * b = f (A3) or b = S[f] (A2), and u = S[S[sigma]] (A3) or S[sigma] (A2).
 * f, u [nrhs][N]: host or device.  info may be NULL.
 * Precision LB_FP32_REFINED runs float32 inner GMRES inside an iterative
 * refinement whose residual b - A sigma (and the potentials giving u) use
 * double-float pair sums.
 * With A3, nrhs >= 2 and any precision but LB_FP64, the right-hand sides
 * are solved in lockstep (groups of up to 64): each GMRES iteration applies
 * A3 to all systems still iterating in one batched pass, and each system
 * stops at its own tolerance; info sums iterations over the right-hand
 * sides and keeps the history of the first.
 * Returns LB_ENOTCONVERGED (with u from the best iterate) when tol is not
 * reached. */
int lb_solve_lb(lb_ctx* ctx, int nrhs, const double* f, double* u, lb_solve_info* info);

/* Harmonic vector fields (Section 5).  For each tangential field F_k
 * (F [nF][N][3], host or device) solve
 *   Delta alpha = div_Gamma F,   Delta beta = -div_Gamma (n x F)
 * as one batch of 2 nF right-hand sides, then
 *   H_k = F_k - grad_Gamma alpha - n x grad_Gamma beta
 * and write H [2 nF][N][3] = (H_1, n x H_1, H_2, n x H_2, ...).  Surface
 * divergence and gradient use nodal differentiation within each patch
 * (Section 2).  info may be NULL. */
int lb_harmonic_fields(lb_ctx* ctx, int nF, const double* F, double* H, lb_solve_info* info);

/* Per-kernel device timing (CUDA events on the context stream) and kernel
 * launch counts, for reporting the split of a solve into its steps.  Not in
 * the paper, whose timings are wall-clock t_q, t_mv, t_s (Section 6). */
#define LB_PROF_FAR32_K1 0     /* float32 charge potential + gradient (S, S', A3 pass 1) */
#define LB_PROF_FAR32_KALL 1   /* float32 S, D, S', S''+D' of one density (A2 pass 1) */
#define LB_PROF_FAR32_K2 2     /* float32 A3 pass 2 */
#define LB_PROF_FAR32_K4 3     /* float32 A2 pass 2 */
#define LB_PROF_FAR64_K1 4     /* the same four in float64 */
#define LB_PROF_FAR64_KALL 5
#define LB_PROF_FAR64_K2 6
#define LB_PROF_FAR64_K4 7
#define LB_PROF_EPILOGUE 8     /* split reduction + near-field correction SpMV */
#define LB_PROF_QUAD 9         /* correction build */
#define LB_PROF_FARDF_K1 10    /* the four pair kernels in double-float arithmetic */
#define LB_PROF_FARDF_KALL 11
#define LB_PROF_FARDF_K2 12
#define LB_PROF_FARDF_K4 13
#define LB_PROF_SHAPE 14       /* node-position gradient pair sums (float64) */
#define LB_PROF_NCAT 16

typedef struct {
  double ms[LB_PROF_NCAT];     /* summed device time per category */
  int64_t calls[LB_PROF_NCAT]; /* timed launches per category */
  int64_t launches;            /* every kernel launched while profiling was on */
  int64_t pairs[LB_PROF_NCAT]; /* far categories: (target, source, density) pair evaluations */
} lb_profile;

/* Turn per-kernel timing on (1) or off (0); either way the counters restart. */
int lb_set_profiling(lb_ctx* ctx, int on);
/* Synchronise the context stream and return the counters since the last
 * lb_set_profiling. */
int lb_get_profile(lb_ctx* ctx, lb_profile* out);

/* Transposed operators of the discrete A3 formulation (float64 pair sums),
 * for density gradients.  The near relation is not symmetric: (S^T y)_j sums
 * over the i with patch(j) not in Near(i) far away and over the transposed
 * correction blocks (Sections 3, 4).  Note that S^T is not the
 * continuous adjoint of S: the discrete matrix carries the quadrature weights
 * of its columns.  y, out [nrhs][N]: host or device.
 * lb_apply_St: out = S^T y.
 * lb_apply_At: out = A^T y for the context's formulation,
 *   A3^T = -I/4 + S'^T S'^T - S^T (S''+D')^T - S^T S'^T 2H + S^T S^T W^T,
 *   A2^T = -I/4 + D^T D^T - (S''+D')^T S^T - S'^T 2H S^T + S^T W^T S^T,
 *   W^T y = w sum(y) / |Gamma|; LB_EINVAL for LB_A1. */
int lb_apply_St(lb_ctx* ctx, int nrhs, const double* y, double* out);
int lb_apply_At(lb_ctx* ctx, int nrhs, const double* y, double* out);

/* Adjoint of lb_solve_lb (not in the paper): the solve is a linear map,
 * u = S S A3^-1 P f (A3) or u = S A2^-1 S P f (A2), P = I - 1 w^T / |Gamma|
 * the weighted mean projection, so the gradient of a loss with respect to f
 * is g_f = P^T A3^-T S^T S^T g_u or P^T S^T A2^-T S^T g_u, with
 * P^T z = z - w sum(z) / |Gamma|.  GMRES on A^T (float64 pairs, the
 * context's tol and max_iter); LB_EINVAL for LB_A1.  g_u, g_f [nrhs][N]: host
 * or device.  info as for lb_solve_lb (may be NULL); LB_ENOTCONVERGED when
 * GMRES does not reach tol. */
int lb_solve_lb_adjoint(lb_ctx* ctx, int nrhs, const double* gu, double* gf, lb_solve_info* info);

/* Gradient of a loss of the A3 solve with respect to the node positions (not
 * in the paper).  The positions enter the discrete A3 operator of Sections 3
 * and 4 only through the far pair sums; the correction weights, the near
 * lists, w, n and H are held fixed.  With A3 sigma = P f, u = S S sigma,
 * z = A3^-T S^T S^T g_u and d = x_i - x_j,
 *   dL = g_u.dS(S sigma) + (S^T g_u).dS(sigma) - z.(dA3 sigma),
 * each term a sum over far pairs of a_i w_j b_j grad_d K(x_i, x_j).(dx_i - dx_j)
 * for K = S, S', S''+D'.  Two GMRES solves (A3 and A3^T, float64 pairs, the
 * context's tol and max_iter) and two float64 gradient pair sums.  f, g_u
 * [nrhs][N], grad [nrhs][N][3]: host or device.  LB_EINVAL unless the
 * formulation is LB_A3; info as for lb_solve_lb (iterations of both solves;
 * may be NULL); LB_ENOTCONVERGED when a GMRES does not reach tol. */
int lb_shape_gradient(lb_ctx* ctx, int nrhs, const double* f, const double* gu, double* grad,
                      lb_solve_info* info);

/* Gradients of a loss of the A3 solve with respect to the surface inputs of
 * lb_upload_geometry (not in the paper): node positions X and chart tangents
 * X_u, X_v, taken as independent inputs, with the correction blocks and the
 * near lists held fixed (they are built once from the geometry and reused).
 *   gX: as lb_shape_gradient (X enters through the far pair sums);
 *   gXu, gXv: X_u and X_v enter through the unit normals
 *     n = X_u x X_v / |X_u x X_v| (target normal of S' and S''+D', source
 *     normal of S''+D'), the weights w = w_ref |X_u x X_v| (every far sum, the
 *     mean W of A3 and the projection P f = f - W f) and the mean curvature
 *     H = -1/2 tr(g^-1 L) with L_ab = X_ab . n and X_uu = D_u X_u,
 *     X_vv = D_v X_v, X_uv = (D_v X_u + D_u X_v)/2 (Sections 2, 4.3).
 * Shares the two float64 GMRES solves (A3 and A3^T) between the outputs.
 * f, g_u [nrhs][N]; gX, gXu, gXv [nrhs][N][3]: host or device, any output may
 * be NULL (gXu and gXv together).  LB_EINVAL unless the formulation is LB_A3,
 * while a far rule is set, or with no output; info as for lb_solve_lb;
 * LB_ENOTCONVERGED when a GMRES does not reach tol. */
int lb_geometry_gradient(lb_ctx* ctx, int nrhs, const double* f, const double* gu, double* gX, double* gXu,
                         double* gXv, lb_solve_info* info);

/* Launch shapes chosen by the batched passes' tuner (not part of the paper;
 * several-density passes time each shape once per process and surface and
 * keep the fastest): shapes[8], indexed by precision (0 float32, 1
 * double-float) * 4 + pass (0: A3 pass 1, 1: pass 2) * 2 + (0: 4 densities,
 * 1: 8 densities per pass).  Values: 0 = 128 threads x 64-source tiles,
 * 1 = 128 x 128, 2 = 256 x 64, -1 = not tuned yet.  shapes[8 + kind], kind
 * 0..3 = K1 (S, grad S), all four kernels, A3 pass 2, A2 pass 2: the
 * variant chosen by timing for single-density float32 passes (K1: 0 scalar
 * with 4 targets per thread, 1 two sources per packed instruction, 2 scalar
 * with 8 targets per thread; the others: 0 packed with 4 targets per thread,
 * 1 the same with registers capped for three resident blocks per SM, 2
 * packed with 2 targets per thread; K1 and A3 pass 2 also 3: each unordered
 * node pair evaluated once for both directions, 4: the same with two
 * sources per packed instruction, 5 and 6: 3 and 4 with two targets per
 * thread), -1 = not tuned yet.  shapes[12], shapes[13]: the symmetric
 * double-float kernels of A3 pass 1 and pass 2 (0: one target per thread,
 * 1: two), -1 = not tuned yet.
 * shapes: host memory of 14 ints. */
int lb_get_tuning(lb_ctx* ctx, int* shapes);

/* Far-field sums of one density that allocate nothing: the float32 pair
 * kernel of lb_far_sums with all of its scratch in a fixed device array that
 * the library carries (12 MiB, held on every GPU that loads the library until
 * the process exits).  The paper has no counterpart; this entry exists for
 * callers that cannot allocate device memory, such as code running inside
 * another runtime's memory pool that owns every allocation on the device, or
 * a service that must keep a fixed device footprint after start-up.  No
 * context is needed.
 *   npatch, np: the surface as for lb_upload_geometry; N = npatch * np must
 *     not exceed 65,536 (LB_EINVAL otherwise, checked without forming the
 *     product; message via lb_last_error(NULL)).
 *   X [N][3], nrm [N][3], w [N]: node positions, unit normals, smooth weights
 *     (device, float64; e.g. from lb_get_geometry).
 *   sigma [N]: the density (device, float64).
 *   row_ptr [N+1], near_patch [nnzb]: the near lists (device; e.g. from
 *     lb_get_corrections); the sums skip exactly those (row, patch) pairs.
 *   out [4][N]: S, D, S', S''+D' far sums (device, float64), as lb_far_sums
 *     with LB_FP32.
 *   stream: cudaStream_t for every launch (NULL = legacy default stream).
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the later calls.  Under CUDA's lazy module
 * loading (the default) that lookup is also when the array is created on the
 * device, so the first call can fail with LB_ECUDA when the device is out of
 * memory: make one call (any valid input) before a memory pool takes the
 * device's memory, and before any stream capture.  Every
 * call shares the one array and overwrites it: calls that may overlap on the
 * GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  Returns LB_ECUDA if the lookup or a launch
 * fails.  No cudaMalloc, cudaFree or allocating library call is made. */
int lb_far_sums_noalloc(int64_t npatch, int np, const double* X, const double* nrm, const double* w,
                        const double* sigma, const int64_t* row_ptr, const int32_t* near_patch,
                        double* out, void* stream);

/* Failure injection for tests (not in the paper): after `after` further
 * device allocations by this context (0 = the very next one), one allocation
 * fails exactly as if cudaMalloc had run out of memory, so the call making it
 * returns LB_ENOMEM; the injection then disarms itself.  after < 0 disarms it.
 * A workspace whose allocation failed is left empty and allocated again by
 * the next call that needs it, so the context stays usable; a failed
 * lb_upload_geometry leaves no geometry (upload again). */
int lb_debug_fail_alloc(lb_ctx* ctx, int64_t after);

/* Launch variant of a timed pass for tests (not in the paper): variant v is
 * used for pass `kind` on this context's surface from now on, in this
 * process, in place of the timed choice.  kind 0..3: the single-density
 * float32 passes (variants as in lb_get_tuning's shapes[8 + kind]); 4, 5: the
 * symmetric double-float kernels of A3 pass 1 and pass 2 (shapes[12],
 * shapes[13]).  LB_EINVAL for a kind or variant out of range (float32
 * variants 3 to 6 exist for kinds 0 and 2 only); LB_ESTATE before a geometry
 * is uploaded. */
int lb_debug_set_variant(lb_ctx* ctx, int kind, int variant);

/* Surface divergence of tangential fields F [nrhs][N][3] -> out [nrhs][N]
 * (Section 2; host or device).  Used for the Hodge right-hand sides and to
 * check harmonic fields (div H = 0). */
int lb_surface_div(lb_ctx* ctx, int nrhs, const double* F, double* out);

/* Octree plan for a fast-multipole far field (host only: no context, no
 * device work; not in the paper, which evaluates its layer potentials with
 * an external FMM library, Section 4.1).  The classical uniform-depth
 * scheme of Greengard and Rokhlin: boxes of level l are the occupied cells
 * of a 2^l grid over a cube holding every node; U(leaf) = the adjacent
 * leaves, itself included; V(box) = the children of the boxes adjacent to
 * its parent that are not adjacent to it (levels >= 2).  For any two
 * leaves exactly one holds: one is in the other's U list, or at exactly
 * one level their ancestors are in each other's V lists.  With a leaf side
 * of at least (near_factor + 1) max_P R_P every near (node, patch) pair lies
 * in adjacent leaves.
 * lb_fmm_plan_create: X [n][3] host float64; the depth is the largest
 *   d <= max_depth (<= 20) whose leaf side (cube side / 2^d) is at least
 *   min_leaf_side.  LB_EINVAL for n < 1, a non-finite coordinate or bad
 *   arguments (message via lb_last_error(NULL)); LB_ENOMEM.
 * lb_fmm_plan_arrays copies (any pointer may be NULL; host int64):
 *   perm [n]: node ids in Morton order (ties by id);
 *   level_ptr [depth+2]: boxes of level l are [level_ptr[l], level_ptr[l+1]);
 *   box_key [nbox]: Morton key (x bit 0, y bit 1, z bit 2, ...) within the
 *     level, ascending per level; box_parent [nbox] (-1 at level 0);
 *   node_ptr [nleaf+1]: leaf b holds perm[node_ptr[b] .. node_ptr[b+1]);
 *   u_ptr [nleaf+1], u_idx [nu]: U lists as leaf indices (b - level_ptr[depth]);
 *   v_ptr [nbox+1], v_idx [nv]: V lists as box indices.
 * The plan owns its arrays until lb_fmm_plan_destroy (accepts NULL). */
typedef struct lb_fmm_plan lb_fmm_plan;
typedef struct {
  int32_t depth;
  int64_t n, nbox, nleaf, nu, nv;
  double lo[3];   /* cube corner */
  double side;    /* cube side */
} lb_fmm_info;
int lb_fmm_plan_create(int64_t n, const double* X, double min_leaf_side, int max_depth, lb_fmm_plan** out);
int lb_fmm_plan_info(const lb_fmm_plan* plan, lb_fmm_info* info);
int lb_fmm_plan_arrays(const lb_fmm_plan* plan, int64_t* perm, int64_t* level_ptr, int64_t* box_key,
                       int64_t* box_parent, int64_t* node_ptr, int64_t* u_ptr, int64_t* u_idx,
                       int64_t* v_ptr, int64_t* v_idx);
int lb_fmm_plan_destroy(lb_fmm_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* GBLB_H */
