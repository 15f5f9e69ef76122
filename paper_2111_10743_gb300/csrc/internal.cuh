// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "gblb.h"

#define LB_PI 3.14159265358979323846
#define LB_INV4PI (1.0 / (4.0 * LB_PI))
#define LB_PINNED_DOUBLES 1024
#define LB_BATCH_MAX 64  // right-hand sides advanced in lockstep by one batched solve

// Device buffer owned by a context; grows on demand and never shrinks.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Far-field kernel variants (which sums a pass accumulates).
enum FarKind {
  FAR_K1 = 0,    // charge q1: potential and gradient           -> S, grad S (S' = n.grad)
  FAR_KALL = 1,  // charge q1: S, D, S', S''+D' of one density   (4 sums)
  FAR_K2 = 2,    // A3 second pass: S'[mu1], S[mu2], S'[mu2], (S''+D')[mu2]
  FAR_K4 = 3,    // A2 second pass: D[mu1], S[mu2]
};

// Cached tile-mask table for one (targets per block, sources per tile) shape.
struct MaskTable {
  int tb = 0, ts = 0;
  int snp = 0;          // source points per patch the table was built for
  int64_t ntb = 0, ntiles = 0;
  uint8_t* flags = nullptr;  // [ntb][ntiles]: 1 when some pair in the block x tile is near
};

struct ProfPending {
  int cat;
  cudaEvent_t a, b;
  int64_t pairs;
};

struct lb_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream for graph captures (made on first use)
  lb_params params{};
  int sm_count = 0;
  std::string err;

  // geometry
  bool have_geom = false;
  int64_t N = 0, npatch = 0;
  int np = 0, order = 0;
  std::vector<double> ref_uv, ref_w;       // host copies of the node rule
  std::vector<double> Vinv, Du, Dv;        // [np][np] host, row-major
  double center[3] = {0, 0, 0};            // mean node position (float32 recentring)
  double df_grid = 0;                      // double-float position grid (power of two)
  double area = 0;

  double* X = nullptr;     // [N][3]
  double* Xu = nullptr;    // [N][3]
  double* Xv = nullptr;    // [N][3]
  double* nrm = nullptr;   // [N][3] unit normals from Xu x Xv
  double* inrm = nullptr;  // [N][3] unit normals of the position interpolant
  double* w = nullptr;     // [N]
  double* H = nullptr;     // [N]
  double* ginv = nullptr;  // [N][3]: g^11, g^12, g^22
  double* J = nullptr;     // [N] |Xu x Xv|
  double* cen = nullptr;   // [npatch][3]
  double* rad = nullptr;   // [npatch]
  double* area_p = nullptr;  // [npatch]
  double* dVinv = nullptr;   // [np][np]
  double* dDu = nullptr;     // [np][np]
  double* dDv = nullptr;     // [np][np]
  double* dref = nullptr;    // [np][3]: u, v, w of the node rule
  float4* pos32 = nullptr;   // [Npad] (x-c, y-c, z-c, 0)
  float4* nrm32 = nullptr;   // [Npad] (nx, ny, nz, 0)
  double4_32a* pos64 = nullptr;  // [Npad] (x, y, z, 0)
  double4_32a* nrm64 = nullptr;  // [Npad] (nx, ny, nz, 0)
  int64_t Npad = 0;

  // near lists and correction blocks
  bool have_near = false, have_corr = false;
  int64_t nnzb = 0;
  int64_t* row_ptr = nullptr;   // [N+1]
  int32_t* near_patch = nullptr;  // [nnzb]
  double* vals = nullptr;       // [nnzb][4][np]
  float* vals_hi = nullptr;     // [nnzb][4][npp] float32 copy (double-float hi part), npp = lb_np_pad(np),
                                // zero past np; made on first use
  float* vals_lo = nullptr;     // [nnzb][4][npp] double-float lo part
  std::vector<MaskTable> masks;
  // transposed near structure (adjoint applies), built on first use
  bool have_trans = false;
  int64_t* tptr = nullptr;                // [npatch+1] per target patch
  int32_t* trow = nullptr;                // [nnzb] rows i with the patch in Near(i), ascending
  int64_t* tblk = nullptr;                // [nnzb] their correction blocks
  unsigned long long* tmask = nullptr;    // [npatch][Npad/64] masked sources per 64-source tile
  uint8_t* tflag = nullptr;               // [target blocks][tiles]
  int64_t t_ntiles = 0, t_ntb = 0;
  double* v0 = nullptr;                   // S^T S^T w
  double* v1 = nullptr;                   // S^T w
  bool adjoint = false;                   // GMRES applies A3^T
  std::map<const void*, int> occupancy;  // resident blocks per SM, per kernel (queried once)

  // profiling
  int prof_on = 0;
  std::vector<ProfPending>* capture_prof = nullptr;  // profiled launches of the graph being captured
  bool capturing = false;                            // a stream capture is in progress
  int64_t launches = 0;
  std::vector<ProfPending> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[LB_PROF_NCAT] = {0};
  int64_t prof_calls[LB_PROF_NCAT] = {0};
  int64_t prof_pairs[LB_PROF_NCAT] = {0};

  // workspace
  DevBuf ws_part, ws_pot, ws_src, ws_vec, ws_red, ws_stage_in, ws_stage_out, ws_gm, ws_quad;
  DevBuf ws_bpot, ws_bgm, ws_bvec;  // batched applies and the lockstep solver
  DevBuf ws_rec;                    // the refinement's recycled Krylov space
  DevBuf ws_dlow;                   // float32 / double-float copies of correction densities
  DevBuf ws_a1;                     // A1 apply: surface gradients and vector single layers
  DevBuf ws_adj;                    // transposed applies
  DevBuf ws_shape, ws_grad;         // node-position gradient: solves, then its pair sums
  double* phi0 = nullptr;           // S[1] for A1's S W S term, in pair precision phi0_prec
  int phi0_prec = -1;
  double* host_pinned = nullptr;  // pinned scalars for GMRES control [LB_PINNED_DOUBLES]
  int64_t fail_alloc_in = -1;     // lb_debug_fail_alloc: device allocations left before a simulated failure

  // oversampled far rule (lb_set_far_rule): Ns = npatch * nps far-field sources
  int far_order = 0, nps = 0;
  int64_t Ns = 0, Nspad = 0;
  std::vector<double> far_uv, far_w;      // host copy of the far rule on T0
  double* fI = nullptr;                   // [nps][np] node-rule Lagrange basis at the far-rule nodes
  double* fY = nullptr;                   // [Ns][3] source positions
  double* fn = nullptr;                   // [Ns][3] unit normals of the interpolated tangents
  double* fw = nullptr;                   // [Ns] weights
  float4* fpos32 = nullptr;               // [Nspad] (y - c, 0), padding far away
  float4* fnrm32 = nullptr;               // [Nspad]
  double4_32a* fpos64 = nullptr;          // [Nspad]
  double4_32a* fnrm64 = nullptr;          // [Nspad]
  DevBuf ws_fden;                         // upsampled densities / target planes
};

// ---- error handling --------------------------------------------------------
int lb_fail(lb_ctx* c, int code, const char* fmt, ...);
#define LB_CUDA(c, expr)                                                              \
  do {                                                                                \
    cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return lb_fail((c), LB_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                     __FILE__, __LINE__);                                             \
  } while (0)
#define LB_CHECK(expr)       \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != LB_OK) return rc_; \
  } while (0)
#define LB_LAUNCH(c)   \
  do {                 \
    ++(c)->launches;   \
    LB_CUDA(c, cudaGetLastError()); \
  } while (0)

// Times the launches enqueued during its lifetime under category `cat` when
// profiling is on (two events recorded on the context stream); `pairs` is the
// number of (target, source, density) pair evaluations they make.
struct ProfScope {
  lb_ctx* c;
  int cat;
  int64_t pairs;
  cudaEvent_t a = nullptr;
  ProfScope(lb_ctx* ctx, int category, int64_t npairs = 0);
  ~ProfScope();
};

// ---- memory ----------------------------------------------------------------
// True when the allocation about to be made must fail (lb_debug_fail_alloc
// armed and counted down to it); disarms itself after firing.
inline bool lb_alloc_fails_now(lb_ctx* c) {
  if (!c || c->fail_alloc_in < 0) return false;
  return c->fail_alloc_in-- == 0;
}
int lb_ensure(lb_ctx* c, DevBuf& b, size_t bytes);
template <typename T>
inline int lb_alloc(lb_ctx* c, T** p, size_t count) {
  if (*p) { cudaFree(*p); *p = nullptr; }
  if (count == 0) return LB_OK;
  if (lb_alloc_fails_now(c))
    return lb_fail(c, LB_ENOMEM, "cudaMalloc(%zu) failed: simulated by lb_debug_fail_alloc", count * sizeof(T));
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) { *p = nullptr; return lb_fail(c, LB_ENOMEM, "cudaMalloc(%zu) failed: %s", count * sizeof(T), cudaGetErrorString(e)); }
  return LB_OK;
}
template <typename T>
inline void lb_free(T** p) {
  if (*p) cudaFree(*p);
  *p = nullptr;
}

// Host-or-device argument staging: returns a device pointer holding `bytes`
// of the caller's data (the caller's own pointer when it is device memory).
int lb_stage_in(lb_ctx* c, const void* src, size_t bytes, DevBuf& tmp, const void** dev);
// For outputs: returns a device pointer to write; lb_stage_out_finish copies
// it back to the caller when the caller passed host memory.
int lb_is_device_ptr(const void* p);
int lb_stage_out(lb_ctx* c, void* dst, size_t bytes, DevBuf& tmp, void** dev);
int lb_stage_out_finish(lb_ctx* c, void* dst, const void* dev, size_t bytes);

// ---- host numerics (node rule matrices) ------------------------------------
int lb_host_basis_matrices(lb_ctx* c);  // fills Vinv, Du, Dv from ref_uv

// ---- internals used across files -------------------------------------------
int lb_require_corr(lb_ctx* c);
int lb_far_launch(lb_ctx* c, int kind, int prec, const void* srcA, const void* srcB,
                  double* part, int* nsplit_out);
// potentials of one density: far + near, writes pot[k][N] for k in `which` bitmask
// (bit K set -> pot + K*N holds K[sigma]); density on device, float64
int lb_potentials(lb_ctx* c, int prec, const double* sigma, double* pot, unsigned which);
// apply the formulation operator to one vector (device in, device out)
int lb_apply_op(lb_ctx* c, int formulation, int prec, const double* tau, double* out);
// A1 applied to one density (device in, device out); leaves S[tau] in ws_pot
int lb_apply_a1(lb_ctx* c, int prec, const double* tau, double* out);
// transposes (float64): A3^T y, S^T y (device in, device out)
int lb_apply_a3t(lb_ctx* c, const double* y, double* out);
int lb_apply_st_dev(lb_ctx* c, const double* y, double* out);
// A3^T or A2^T by the context's formulation
int lb_apply_at_op(lb_ctx* c, const double* y, double* out);
int lb_build_transpose(lb_ctx* c);
// node-position gradient of an A3-solve loss from sigma, S' sigma, S sigma,
// S^T g_u and z = A3^-T S^T S^T g_u (device, float64); grad [N][3]
int lb_shape_grad_pairs(lb_ctx* c, const double* gu, const double* sg, const double* mu1, const double* mu2,
                        const double* q1, const double* z, double* grad);
// gradient with respect to the tangents X_u, X_v (n, w, H through them), from
// the projected right-hand side pf and the same vectors; gXu, gXv [N][3]
int lb_tangent_grad_pairs(lb_ctx* c, const double* gu, const double* pf, const double* sg, const double* mu1,
                          const double* mu2, const double* q1, const double* z, double* gXu, double* gXv);
void lb_free_transpose(lb_ctx* c);
int lb_get_mask(lb_ctx* c, int tb, int ts, MaskTable** out);
// the same for sources of snp points per patch padded to nsrc_pad (the
// oversampled far rule)
int lb_get_mask_src(lb_ctx* c, int tb, int ts, int snp, int64_t nsrc_pad, MaskTable** out);
// oversampled far rule: sources for a pass (as pack_sources), and its state
int lb_far_rule_pack(lb_ctx* c, int prec, const double* d1, const double* d2, void** A, void** B);
void lb_free_far_rule(lb_ctx* c);
// float32 hi / lo copies of the correction weights (no-op when present)
int lb_lowp_vals(lb_ctx* c);
// hi[i] = (float)x[i], lo[i] = (float)(x[i] - hi[i]) (lo may be null)
int lb_split_f64(lb_ctx* c, int64_t n, const double* x, float* hi, float* lo);
int lb_pack_df(lb_ctx* c, const double* d1, const double* d2, void* S);
int lb_pack_df_points(lb_ctx* c, int64_t n, int64_t npad, const double* Y, const double* nY, const double* wY,
                      const double* d1, const double* d2, void* S);
// Double-float pass of `kind` over the packed planes S.  *nsplit > 0: part
// holds nsplit split partials [nsplit][4][N] of (hi, lo) float pairs;
// *nsplit == -1: part holds one float64 sum per accumulator, [4][N] (the
// symmetric kernel of the node-source passes K1 and K2).
int lb_far_launch_df(lb_ctx* c, int kind, const void* S, double* part, int* nsplit);
// launch variant chosen for single-density float32 passes of `kind`, -1 if not tuned yet
int lb_far_tuned_variant(lb_ctx* c, int kind);
// Timing-based choice among nvar launch variants of one pass (launch(c, v,
// arg) runs variant v): each is launched twice, the second timed, once per
// (device, N, n_p, key_kind) and process; the fastest is kept.  Variant 0
// while a graph is being captured and nothing is tuned yet.  key_kind 0..3:
// the float32 single-density kinds; LB_TUNE_DFSYM + kind: the symmetric
// double-float kernels.
#define LB_TUNE_DFSYM 8
int lb_tune_choice(lb_ctx* c, int key_kind, int nvar, int (*launch)(lb_ctx*, int, void*), void* arg, int* choice);
// the choice made for key_kind, -1 if not tuned yet
int lb_tuned_choice(lb_ctx* c, int key_kind);
// A3 applied to R densities tau[R][N] -> out[R][N] with several densities per
// far-field pass (prec LB_FP32 or LB_DF64); u (may be null) receives S[S[tau]]
int lb_apply_a3_batch(lb_ctx* c, int prec, int R, const double* tau, double* out, double* u);
// S applied to R densities sig[R][N] -> out[R][N] (far + near)
int lb_apply_s_batch(lb_ctx* c, int prec, int R, const double* sig, double* out);
// weighted mean of a device vector (deterministic), result to host
int lb_wmean(lb_ctx* c, const double* f, double* mean_host);
// counters of the last solve
extern thread_local int64_t lb_pair_counter;
extern thread_local int lb_apply64_counter, lb_apply32_counter;
extern thread_local int lb_graph_counter;  // GMRES iterations run as graph replays

static inline unsigned lb_div_up(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }
// Source-split count for a pair kernel launched as ntb target blocks x
// nsplit source ranges of ntiles tiles: the smallest split (at most 32) whose
// grid fills whole waves of the kernel's resident blocks to >= 97%, else the
// best fill found.  The resident-block count is queried once per kernel, so
// the launches of a captured iteration make no queries.
template <typename F>
int lb_pick_nsplit(lb_ctx* c, F kernel, int nth, int64_t ntb, int64_t ntiles, int* out) {
  int per_sm = 0;
  auto it = c->occupancy.find((const void*)kernel);
  if (it != c->occupancy.end()) {
    per_sm = it->second;
  } else {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nth, 0);
    if (e != cudaSuccess) return lb_fail(c, LB_ECUDA, "occupancy query failed: %s", cudaGetErrorString(e));
    c->occupancy[(const void*)kernel] = per_sm;
  }
  const int64_t slots = (int64_t)(per_sm > 0 ? per_sm : 1) * c->sm_count;
  int best = 1;
  double best_eff = -1;
  const int64_t hi = ntiles < 32 ? ntiles : 32;
  for (int64_t s = 1; s <= hi; ++s) {
    const int64_t tps = (ntiles + s - 1) / s;
    const int64_t ns = (ntiles + tps - 1) / tps;
    const int64_t blocks = ntb * ns;
    const double waves = (double)blocks / (double)slots;
    const double eff = waves / std::ceil(waves);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = (int)ns;
    }
    if (eff > 0.97 && blocks >= slots) break;
  }
  *out = best;
  return LB_OK;
}

// nodes per patch rounded up to a multiple of four: row length of the float
// copies of the correction weights and densities (16-byte loads)
static inline int lb_np_pad(int np) { return (np + 3) & ~3; }
