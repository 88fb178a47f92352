/*
 * ccladder.h -- C ABI of the GB300 (sm_103a) CD-CCSD vvvv ladder library.
 *
 * Closed-shell problem statement (arXiv:2202.02019):
 *   Cholesky integrals (Sec. II.A):        g_acbd = sum_J L^J_ac L^J_bd
 *   ladder amplitudes:                      tau_ij^cd = t_ij^cd + t_i^c t_j^d
 *   ladder residual (Sec. II.B, A2 term):   Omega_ij^ab = sum_cd g_acbd tau_ij^cd
 *   V^4 density (Eq. v4density, App. A):    Gamma_abcd = sum_ij tbar_ij^ab tau_ij^cd
 *   three-index density (Sec. II.C, the V^4 part of W-tilde, built with L):
 *                                           D^J_ac = sum_bd Gamma_abcd L^J_bd
 *   Lagrangian slice (Eq. lagrangian):      E = sum_ijab tbar_ij^ab Omega_ij^ab
 * D carries no factor 2: Eq. (integral_contraction) has the 2, so dE/dL = 2 D.
 * Neither g nor Gamma is ever stored whole: both are built in tiles of
 * virtual-pair blocks and consumed at once (Sec. II.B / App. A storage policy),
 * using the symmetric/antisymmetric pair packing of Sec. II.B.
 *
 * Conventions shared by every entry point
 *   - All array arguments are DEVICE pointers to float64, C-contiguous:
 *       L_vv  [nj][v][v]    L^J_ac   at (J*v + a)*v + c
 *       t1    [o][v]        t_i^a    (may be NULL: tau = t2)
 *       t2    [o][o][v][v]  t_ij^ab  at ((i*o + j)*v + a)*v + b
 *       tbar2 [o][o][v][v]  same layout as t2
 *       eps   [o + v]       orbital energies, occupied first
 *       omega [o][o][v][v]  output, same layout as t2
 *       D     [nj][v][v]    output, same layout as L_vv
 *     Kernels do not assume L^J symmetric.  t2 and tbar2 MUST be pair
 *     symmetric (t_ij^ab = t_ji^ba); the packed algorithm relies on it.
 *   - Outputs are overwritten, never accumulated into.  The library keeps no
 *     pointer after return and never allocates or frees device memory: the
 *     caller owns every buffer, including the workspace `ws` (device, 256-byte
 *     aligned, at least cc_ladder_workspace_size() bytes).  Calls that share
 *     a workspace must be ordered on one stream.
 *   - `stream` is a cudaStream_t (NULL: legacy default stream).  Calls are
 *     asynchronous.  Calls that compute both Omega and D (cc_ladder_step,
 *     cc_ladder_step_blocks) run the density chain on one internal stream per
 *     device, created on the first such call with that device current (make
 *     it before any stream capture), forked from `stream` after the
 *     preparation and joined back to it before the call's last kernels; work
 *     enqueued on `stream` afterwards sees all of the call's results.
 *     Host-detectable argument errors are returned at once,
 *     device-side errors (bounded waits that gave up) are latched in the
 *     workspace and reported by cc_ladder_status().  Each call clears the
 *     latched status at its start, so read it after the call it concerns.
 *   - n_sys > 1 runs independent systems on `stream`.  With a workspace of
 *     cc_ladder_workspace_size(sys, n_sys, p, which) bytes they run back to
 *     back, sharing it.  With at least cc_ladder_workspace_size(sys, n_sys, p,
 *     which | CC_WS_BATCH) bytes (each system's prepared operands plus
 *     scratch for up to 8 pair blocks in flight) the batched schedule runs
 *     instead: every contraction launch carries pair blocks of up to 8
 *     systems, the ones with the most work left, pulled tile by tile from a
 *     device queue.  Both give the same bits for the split precisions: every
 *     output tile is computed the same way, and each system's pair blocks
 *     keep their order.
 *   - Return codes: 0 or a negative CC_ERR_* value; no host aborts, no
 *     exceptions across the ABI.
 */
#ifndef CCLADDER_H
#define CCLADDER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CC_PREC_FP64 = 0,   /* FP64 operands, FP64 DMMA tensor-core products          */
  CC_PREC_MIXED = 1,  /* 3-piece split-BF16 operands (24 bits), 6 tcgen05 products
                         per useful product, FP32 tensor-core accumulation in
                         restarted windows summed error-free, float-float
                         intermediates, FP64 outputs and reductions            */
  CC_PREC_FP16X2 = 2  /* as CC_PREC_MIXED with 2-piece split-FP16 operands
                         (22 bits) scaled per matrix by a power of two, 3
                         products per useful product: half the tensor work     */
} cc_precision;

enum {
  CC_OK = 0,
  CC_ERR_ARG = -1,        /* NULL pointer, dims < 1, misaligned, bad n_sys     */
  CC_ERR_DEVICE = -2,     /* current device is not sm_103                      */
  CC_ERR_WORKSPACE = -3,  /* ws_bytes smaller than cc_ladder_workspace_size()  */
  CC_ERR_CUDA = -4,       /* a CUDA call or launch failed (see strerror)       */
  CC_ERR_TIMEOUT = -5,    /* a bounded device wait gave up                     */
  CC_ERR_SIZE = -6        /* request larger than a fixed-size device scratch   */
};

/* which-flags for cc_ladder_workspace_size.  CC_WS_BATCH, or-ed with the
 * others, asks for the size of the batched schedule (see n_sys above). */
enum {
  CC_WS_RESIDUAL = 1,
  CC_WS_DENSITY = 2,
  CC_WS_LAGRANGIAN = 4,
  CC_WS_STEP = 7,
  CC_WS_BATCH = 8
};

typedef struct {
  int32_t o, v, nj;       /* occupied, virtual, Cholesky vectors; all >= 1      */
  const double* L_vv;     /* [nj][v][v]                                         */
  const double* t1;       /* [o][v] or NULL                                     */
  const double* t2;       /* [o][o][v][v], pair symmetric                       */
  const double* tbar2;    /* [o][o][v][v], pair symmetric; density/lagrangian   */
  const double* eps;      /* [o+v]; only cc_ladder_update reads it              */
} cc_ladder_system;

/* Bytes of workspace needed by the calls selected in `which` (CC_WS_* bits)
 * for this list of systems at precision p.  0 on invalid arguments. */
size_t cc_ladder_workspace_size(const cc_ladder_system* sys, int n_sys,
                                cc_precision p, int which);

/* Ladder residual Omega_ij^ab = sum_cd g_acbd tau_ij^cd (Sec. II.B).
 * omega[s] is a device [o][o][v][v] buffer per system. */
int cc_ladder_residual(const cc_ladder_system* sys, int n_sys,
                       double* const* omega, cc_precision p,
                       void* ws, size_t ws_bytes, void* stream);

/* Adjoint ladder: out_ij^cd = sum_ab tbar_ij^ab g_acbd = dE/dtau_ij^cd, the
 * derivative of E = sum tbar . Omega with respect to the ladder amplitudes
 * (Omega is linear in tau).  Computed as the ladder with L^J_ac replaced by
 * L^J_ca applied to tbar2 (t1 and t2 are not read), so the g tiles are
 * rebuilt, never stored.  out[s] is a device [o][o][v][v] buffer; requires
 * tbar2.  Workspace: CC_WS_RESIDUAL. */
int cc_ladder_residual_adjoint(const cc_ladder_system* sys, int n_sys,
                               double* const* out, cc_precision p,
                               void* ws, size_t ws_bytes, void* stream);

/* Three-index density D^J_ac = sum_bd Gamma_abcd L^J_bd with
 * Gamma_abcd = sum_ij tbar_ij^ab tau_ij^cd (Eq. v4density of Sec. II.B; D is the
 * V^4 part of the W-tilde intermediate of Sec. II.C).
 * D[s] is a device [nj][v][v] buffer per system; requires tbar2. */
int cc_ladder_density(const cc_ladder_system* sys, int n_sys,
                      double* const* D, cc_precision p,
                      void* ws, size_t ws_bytes, void* stream);

/* Excited-state V^4 density intermediate (App. A: d^es_abcd = O^(2)_abcd(L2, U)
 * with U = T2 R0 + R2), in the T1-transformed basis:
 *     D^J_ac = sum_bd Gamma_abcd L^J_bd,  Gamma_abcd = sum_ij L2_ij^ab U_ij^cd,
 *     U_ij^cd = R0[s] * t2_ij^cd + R2[s]_ij^cd.
 * sys[s].tbar2 holds the left doubles L2, sys[s].t2 the ground-state doubles
 * T2 and L_vv the (T1-transformed) Cholesky vectors; sys[s].t1 is not read.
 * R2[s] is a device [o][o][v][v] buffer (pair symmetric, like t2); R0 is a
 * HOST array of n_sys doubles.  D[s] as for cc_ladder_density; workspace:
 * CC_WS_DENSITY. */
int cc_ladder_density_es(const cc_ladder_system* sys, int n_sys,
                         const double* const* R2, const double* R0,
                         double* const* D, cc_precision p,
                         void* ws, size_t ws_bytes, void* stream);

/* E[s] = sum_ijab tbar_ij^ab Omega_ij^ab (Eq. lagrangian, the ladder slice),
 * an FP64 reduction written to the device array E[n_sys].  If omega_opt is
 * non-NULL its buffers hold Omega already (from cc_ladder_residual); if NULL
 * Omega is computed internally into workspace.  Requires tbar2. */
int cc_ladder_lagrangian(const cc_ladder_system* sys, int n_sys, double* E,
                         double* const* omega_opt, cc_precision p,
                         void* ws, size_t ws_bytes, void* stream);

/* One whole pass: Omega, D and E from one shared preparation of L, tau and
 * tbar (the three calls above fused).  Workspace: CC_WS_STEP. */
int cc_ladder_step(const cc_ladder_system* sys, int n_sys,
                   double* const* omega, double* const* D, double* E,
                   cc_precision p, void* ws, size_t ws_bytes, void* stream);

/* Sharding a system over several GPUs (pair blocks, the virtual-pair
 * blocking of Sec. II.B's restricted loops a <= b: block (alpha <= beta)
 * holds the pairs a <= b with a in virtual-row block alpha and b in block
 * beta, blocks of `edge` rows, numbered alpha-major, beta = alpha .. last).
 * cc_ladder_pair_blocks returns their number and the edge for this system
 * under the current tuning (host only, no device work).
 * cc_ladder_step_blocks runs cc_ladder_step restricted to the n_blocks
 * distinct pair blocks listed in the HOST array `blocks`:
 *   omega   [o][o][v][v]  Omega_ij^ab and Omega_ij^ba for the pairs a <= b of
 *                         those blocks (other elements are not touched);
 *   D_part  [nj][v][v]    the contribution of those blocks to D (overwritten);
 *   E_part  [1]           sum over those blocks' pairs of tbar . Omega.
 * Over a partition of the blocks the omegas are disjoint and complete, and
 * the D_part and E_part sum to D and E (up to the order of the additions: a
 * multi-GPU run finishes D with one reduce-scatter and E with one all-reduce).
 * The outputs of a pair block do not depend on the other blocks of the list:
 * on the split precisions a shard's omega entries are the same bits as those
 * of cc_ladder_step (the FP64 path adds split-K chunks with atomics, so there
 * they agree up to the order of those additions).
 * Workspace: CC_WS_STEP for this one system; n_sys is 1. */
int cc_ladder_pair_blocks(const cc_ladder_system* sys, int32_t* count, int32_t* edge);
int cc_ladder_step_blocks(const cc_ladder_system* sys, const int32_t* blocks, int n_blocks,
                          double* omega, double* D_part, double* E_part, cc_precision p,
                          void* ws, size_t ws_bytes, void* stream);

/* Jacobi amplitude step t'_ij^ab = t_ij^ab + Omega_ij^ab /
 * (eps_i + eps_j - eps_a - eps_b), in FP64 (the paper leaves the solver
 * step unstated; this is the orbital-energy-denominator update).
 * t2_out may equal sys->t2 only if no other call still reads it. */
int cc_ladder_update(const cc_ladder_system* sys, int n_sys,
                     double* const* omega, double* const* t2_out,
                     void* stream);

/* T1-transformed Cholesky vectors, virtual-virtual block (Sec. II.C: the
 * integrals and Cholesky vectors in the T1-transformed basis, x = I - t1,
 * y = I + t1^T, L^J -> x L^J y^T):
 *     L_vv_t1[J][a][c] = L_vv[J][a][c] - sum_i t1[i][a] * L_ov[J][i][c]
 * In that basis the ladder takes t2 itself: run the calls above with
 * L_vv = L_vv_t1 and t1 = NULL (the kernels do not assume L^J symmetric).
 * L_ov [nj][o][v] is the occupied-virtual block of the MO Cholesky vectors,
 * L^J_ic at (J*o + i)*v + c; t1 [o][v]; L_vv_t1 [nj][v][v], must not overlap
 * an input.  FP64 throughout.  Device pointers; asynchronous on `stream`. */
int cc_ladder_t1_transform(int32_t o, int32_t v, int32_t nj, const double* L_vv,
                           const double* L_ov, const double* t1, double* L_vv_t1,
                           void* stream);

/* Back-transformation of a three-index density intermediate to the MO
 * basis (Sec. II.C: (W^J)^MO = x^T W^J y) for a W^J that is non-zero in
 * the virtual-virtual block only, such as D from cc_ladder_density in the
 * T1 basis.  The vv block is unchanged; the occupied-virtual block is
 *     W_ov[J][i][c] = - sum_a t1[i][a] * W_vv[J][a][c]
 * W_vv [nj][v][v], t1 [o][v], W_ov [nj][o][v] (output, must not overlap an
 * input).  FP64.  Device pointers; asynchronous on `stream`. */
int cc_ladder_w_backtransform(int32_t o, int32_t v, int32_t nj, const double* W_vv,
                              const double* t1, double* W_ov, void* stream);

/* Ground-state OV^3 density contributions to the three-index intermediates
 * (Sec. II.C with App. A: d_abci = 0 and d_abic = L^a_m t~^cb_im R0 in the
 * ground state, t~_ij^ab = 2 t_ij^ab - t_ji^ab), built without the OV^3 array
 * through the intermediates of Table I, with L^K in place of Z^K (as for D):
 *     W_vv[K][a][b] = R0 sum_m tbar1[m][a] Y~^K_bm,   Y~^K_bm = sum_ic t~^cb_im L^K_ic
 *     W_ov[K][i][c] = R0 sum_mb t~^cb_im O^K_bm,      O^K_bm  = sum_a tbar1[m][a] L^K_ab
 * tbar1 [o][v] holds the singles multipliers L^a_m at m*v + a; t2 [o][o][v][v]
 * (pair symmetric); L_vv [nj][v][v]; L_ov [nj][o][v].  Outputs are
 * overwritten: W_vv [nj][v][v], W_ov [nj][o][v].  The two (o v) x N_J
 * contractions run on FP64 DMMA for CC_PREC_FP64 and on split BF16 for either
 * split precision; the small ones in FP64.  Workspace:
 * cc_ladder_ov3_workspace_size() bytes, 256-byte aligned. */
size_t cc_ladder_ov3_workspace_size(int32_t o, int32_t v, int32_t nj, cc_precision p);
int cc_ladder_ov3_gs(int32_t o, int32_t v, int32_t nj, const double* L_vv, const double* L_ov,
                     const double* t2, const double* tbar1, double R0, double* W_vv,
                     double* W_ov, cc_precision p, void* ws, size_t ws_bytes, void* stream);

/* Excited-state d_abci block (App. A: d^es_abci = L_ji^ac R_j^b) and its
 * contributions to the three-index intermediates (Sec. II.C, Table I), again
 * without the OV^3 array and with L^K in place of Z^K:
 *     W_vv[K][a][b] = sum_j R_j^b X^K_aj,   X^K_aj = sum_ic L_ji^ac L^K_ic
 *     W_vo[K][i][c] = W_ci^K = sum_aj L_ji^ac P^K_aj,   P^K_aj = sum_b R_j^b L^K_ab
 * L2 [o][o][v][v] holds the left doubles (L_ij^ab at ((i*o + j)*v + a)*v + b,
 * pair symmetric); R1 [o][v] the right singles (R_j^b at j*v + b).  Outputs
 * overwritten.  Precision, workspace (cc_ladder_ov3_workspace_size) and
 * arithmetic as for cc_ladder_ov3_gs. */
int cc_ladder_ov3_es_abci(int32_t o, int32_t v, int32_t nj, const double* L_vv, const double* L_ov,
                          const double* L2, const double* R1, double* W_vv, double* W_vo,
                          cc_precision p, void* ws, size_t ws_bytes, void* stream);

/* Excited-state d_abic block (App. A, eight terms, taken as printed):
 *   d^es_abic = L^a_m t~^cb_im R0 + L^a_m (2 R~^bc_mi - R~^cb_mi) + 2 X_ab R^c_i
 *             - (V_akbi + Y_akbi) R^c_k + L^ad_mk t~^bc_mi R^d_k - L^ad_mn t^bc_mn R^d_i
 *             + Y~_akci R^b_k - X_ac R^b_i
 * with X_ab = L^ad_kl t^bd_kl, Y_ajbi = L^ad_jl t^bd_il, V_ajbi = L^ac_kj t^bc_ki,
 * Y~_djak = L^ed_mj t~^ea_mk (Table I, App. A), t~ = 2 t_ij - t_ji and R~ likewise,
 * and its contributions to the three-index intermediates (Sec. II.C), L^K in
 * place of Z^K, never forming the OV^3 array:
 *     W_vv[K][a][b] = sum_ic d_abic L^K_ic,   W_ov[K][i][c] = sum_ab d_abic L^K_ab.
 * tbar1 [o][v] = L^a_m (left singles), L2 [o][o][v][v] (left doubles) and
 * t2, R2 [o][o][v][v] pair symmetric, R1 [o][v] = R_i^a; outputs overwritten.
 * The large contractions run on the FP64 DMMA engine for CC_PREC_FP64 and on
 * split BF16 for either split precision, the thin ones in FP64.  Workspace:
 * cc_ladder_ov3_es_abic_workspace_size() bytes, 256-byte aligned (it holds
 * the O^2V^2 intermediates V + Y and Y~, (o v)^2 doubles each). */
size_t cc_ladder_ov3_es_abic_workspace_size(int32_t o, int32_t v, int32_t nj, cc_precision p);
int cc_ladder_ov3_es_abic(int32_t o, int32_t v, int32_t nj, const double* L_vv, const double* L_ov,
                          const double* tbar1, const double* L2, const double* t2, double R0,
                          const double* R1, const double* R2, double* W_vv, double* W_ov,
                          cc_precision p, void* ws, size_t ws_bytes, void* stream);

/* MP2-like driver of the doubles equations from the occupied-virtual block
 * of the Cholesky vectors (Sec. II.A):
 *     g[i][j][a][b] = g_aibj = sum_J L^J_ia L^J_jb      (t2 layout, [o][o][v][v])
 * L_ov [nj][o][v] (L^J_ia at (J*o + i)*v + a, symmetric MO vectors: L_ai = L_ia).
 * An o v x o v contraction over J: FP64 DMMA for CC_PREC_FP64, split BF16
 * (float-float result) for either split precision.  The output is made
 * exactly pair symmetric (g_aibj = g_bjai).  Workspace: at least
 * cc_ladder_mp2_driver_workspace_size() bytes, 256-byte aligned. */
size_t cc_ladder_mp2_driver_workspace_size(int32_t o, int32_t v, int32_t nj, cc_precision p);
int cc_ladder_mp2_driver(int32_t o, int32_t v, int32_t nj, const double* L_ov, double* g,
                         cc_precision p, void* ws, size_t ws_bytes, void* stream);

/* n_iter Jacobi steps of the doubles amplitude equations restricted to the
 * ladder and the MP2-like driver (the CC equations of Sec. II.A solved with
 * the orbital-energy denominators; the paper leaves the solver to its CC
 * program):
 *     t' = (g_aibj + (Omega_ij^ab + Omega_ji^ba) / 2) / (eps_i + eps_j - eps_a - eps_b),
 *     Omega = sum_cd g_acbd tau_ij^cd,  tau = t + t1 (x) t1 with sys->t1 fixed.
 * sys: L_vv, t1 (may be NULL), t2 = the starting amplitudes (read only),
 * eps (required).  g_drv: device [o][o][v][v] driver (cc_ladder_mp2_driver).
 * The final amplitudes go to t2_out (may equal sys->t2); dnorm2 is a device
 * array of n_iter doubles receiving sum (t' - t)^2 of each step.  One
 * system per call.  Workspace: cc_ladder_iterate_workspace_size() bytes
 * (the residual's workspace plus two [o][o][v][v] FP64 buffers).  The
 * latched status (cc_ladder_status) covers all steps of the call. */
size_t cc_ladder_iterate_workspace_size(const cc_ladder_system* sys, cc_precision p);
int cc_ladder_iterate(const cc_ladder_system* sys, const double* g_drv, int n_iter,
                      double* t2_out, double* dnorm2, cc_precision p,
                      void* ws, size_t ws_bytes, void* stream);

/* x[k] *= factor * g[0] for k < n, on the device (g: a device double, or NULL
 * for 1).  The chain rule of the differentiable energy: dE/dL = 2 D times the
 * incoming gradient of E (Eq. integral_contraction carries the 2), dE/dtau
 * and dE/dtbar times that gradient, without a host round trip. */
int cc_ladder_scale_by(double* x, int64_t n, double factor, const double* g, void* stream);

/* Synchronises `stream`, then returns and clears the device-side status
 * latched in `ws` by earlier calls (CC_OK or CC_ERR_TIMEOUT), or
 * CC_ERR_CUDA if the stream reports an error. */
int cc_ladder_status(void* ws, void* stream);

/* Same value as cc_ladder_lagrangian with omega_opt given, for callers that
 * cannot allocate device memory where they need E (a solver loop inside
 * another framework's memory pool, or one that must not pay cudaMalloc's
 * implicit synchronisation): no workspace argument and no allocation.  The
 * paper has no counterpart; this is a library convenience.
 * The partial sums live in a fixed device array of the library
 * (64 systems x 1024 doubles = 512 KiB, held on every GPU that loads the
 * library until the process exits).  At most 64 systems per call; more
 * returns CC_ERR_SIZE.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current; under
 * CUDA's lazy module loading that is also when the driver brings this part of
 * the library, array included, onto the GPU.  Make that first call before any
 * stream capture and before relying on the device's free memory staying put;
 * later calls allocate nothing.  All calls share the array and it
 * keeps the last call's contents (each call overwrites what it reads);
 * calls that overlap on the GPU -- other streams, other host threads on the
 * same device -- race on it and must be serialised by the caller. */
int cc_ladder_lagrangian_noalloc(const cc_ladder_system* sys, int n_sys, double* E,
                                 double* const* omega, void* stream);

/* Testing hook for the bounded-wait machinery: launches one kernel that
 * spins on the device int *flag until it becomes non-zero or `timeout_ns`
 * nanoseconds pass; on timeout it latches CC_ERR_TIMEOUT in `ws` and
 * returns.  Read the outcome with cc_ladder_status(). */
int cc_ladder_debug_wait(const int* flag, long long timeout_ns, void* ws,
                         void* stream);

/* Static description of a return code; for CC_ERR_CUDA the text of the
 * last CUDA error seen by the library is appended. */
const char* cc_ladder_strerror(int code);

/* Tuning knobs, process-wide, for calls made afterwards (0 = default):
 *   block_edge   virtual rows per pair block (multiple of 4, <= 256; default
 *                48).  Sets the scratch size: size workspaces after changing it.
 *   win_kblocks  split paths, CC_KERNEL_SINGLE and CC_KERNEL_PAIR kernels: the
 *                leading-piece product is re-started every win_kblocks * 32
 *                K-terms, rounded down to the contraction's 64-term K step and
 *                at least one step, so 1 and 2 give the same window (1, 2, 4
 *                or 8; default 4 for CC_PREC_MIXED, 2 for CC_PREC_FP16X2).
 *                The CC_KERNEL_KBLOCK_WINDOWS kernel (the CC_PREC_FP16X2
 *                default) has one window per k-block and ignores it.
 *                The split paths' error is proportional to the window
 *                (retinal-scale system, split BF16, E against the FP64 path:
 *                1.8e-7 at 2, 3.5e-7 at 4, 7.2e-7 at 8); 8 can exceed 1e-6
 *                (1.09e-6 for Omega at o=6, v=157, N_J=300), and so can 4 on
 *                CC_PREC_FP16X2 with the single-CTA kernel (1.01e-6 at o=6,
 *                v=61, N_J=305).
 * Returns CC_ERR_ARG for other values.  Not synchronised with calls in flight
 * on other host threads. */
int cc_ladder_set_tuning(int block_edge, int win_kblocks);

/* Which tensor-core contraction kernel the split paths use, process-wide, for
 * calls made afterwards:
 *   0                 default: CC_KERNEL_SINGLE for CC_PREC_MIXED,
 *                     CC_KERNEL_KBLOCK_WINDOWS for CC_PREC_FP16X2;
 *   CC_KERNEL_SINGLE  one CTA per 128 x 128 output tile;
 *   CC_KERNEL_PAIR    a cluster of two CTAs per 256 x 128 output tile
 *                     (tcgen05.mma.cta_group::2: each CTA loads its 128 rows of
 *                     A and half of B; 25 % fewer operand bytes per SM and a
 *                     deeper load pipeline);
 *   CC_KERNEL_KBLOCK_WINDOWS  one CTA per 128 x 128 tile, every 64-term
 *                     k-block its own window holding all its products (the
 *                     small ones first), three window buffers, one commit per
 *                     k-block; the window knob does not apply;
 *   CC_KERNEL_PAIR_KBLOCK_WINDOWS  the CTA-pair tiles with one window per
 *                     k-block (three window buffers, three stages).
 * SINGLE and PAIR form every output element from the same products, windows
 * and folds (bit-identical results), and so do the two KBLOCK_WINDOWS kinds;
 * the two groups round differently.
 * Returns CC_ERR_ARG for other values.  Not synchronised with calls in flight
 * on other host threads. */
#define CC_KERNEL_SINGLE 1
#define CC_KERNEL_PAIR 2
#define CC_KERNEL_KBLOCK_WINDOWS 3
#define CC_KERNEL_PAIR_KBLOCK_WINDOWS 4
int cc_ladder_set_contraction(int kind);

/* Kernel launches issued by the calls above since the library was loaded
 * (a host-side counter). */
long long cc_ladder_launch_count(void);

/* Instrumentation (not part of the paper's method).  cc_ladder_profile(1)
 * makes every later call record a CUDA event pair on its stream around each
 * tensor-core contraction launch; cc_ladder_profile_read() waits for the
 * recorded events and returns the contraction time in milliseconds (the length
 * of the union of the launches' intervals: launches on the library's second
 * stream may overlap those on the caller's),
 * the number of contraction launches and their padded 2*M*N*K flop count,
 * then clears them.  cc_ladder_profile(0) switches recording off. */
void cc_ladder_profile(int enable);
int cc_ladder_profile_read(double* gemm_ms, long long* gemm_launches, double* gemm_flops);

#ifdef __cplusplus
}
#endif
#endif /* CCLADDER_H */
