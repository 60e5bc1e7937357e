/*
 * dwfmg.h -- C ABI of the GB300 (sm_103a) domain wall fermion multigrid hot path.
 *
 * Operators and algorithms: Boyle & Yamaguchi, "Comparison of Domain Wall
 * Fermion Multigrid Methods", arXiv:2103.05034.
 *
 * ---------------------------------------------------------------------------
 * Conventions shared by every call
 * ---------------------------------------------------------------------------
 * Lattice.  L[4] = {Lx, Ly, Lz, Lt}, each even; fifth dimension Ls in
 *   {4, 8, 16, 24}.  Periodic boundaries in all four directions.  A 4D site
 *   (x,y,z,t) has lexicographic index i4 = x + Lx*(y + Ly*(z + Lz*t)) and
 *   parity (x+y+z+t) mod 2 (0 = even).  Vh = Lx*Ly*Lz*Lt/2 sites per parity;
 *   the checkerboard index of a site is i4/2.
 *
 * Spin basis.  Chiral: gamma_k = [[0,-i sigma_k],[i sigma_k,0]] (k = x,y,z),
 *   gamma_t = [[0,1],[1,0]], gamma_5 = gamma_x gamma_y gamma_z gamma_t =
 *   diag(1,1,-1,-1); P_+- = (1 +- gamma_5)/2.
 *
 * Gauge field (input to dwf_ctx_create).  complex128, [T][Z][Y][X][mu][3][3],
 *   mu = 0..3 is x,y,z,t, row-major colour matrices; U_mu(x) transports from
 *   x+mu to x as in Eq. (2).  Host or device memory.
 *
 * Fermion fields (every other buffer).  Device memory unless a call says
 *   otherwise.  Complex numbers are (re, im) pairs of the element type of the
 *   precision argument:
 *     DWF_F64  double   (16 bytes per complex)
 *     DWF_F32  float    (8 bytes per complex)
 *     DWF_F16S half     (4 bytes per complex; arithmetic is FP32)
 *   A half field (one parity) is [Vh][spin 4][colour 3][Ls]: the fifth
 *   dimension is innermost.  A full field is [parity 2][Vh][4][3][Ls] (the
 *   even half first).  A batch of nrhs fields is nrhs such fields back to
 *   back.  Buffers must be 16-byte aligned and must not overlap unless a call
 *   says otherwise.
 *
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *   are asynchronous on that stream unless they return results to the host
 *   (solvers, power method, setup), which synchronise once before returning.
 *
 * Ownership.  The caller owns every field buffer.  The library owns
 *   dwf_ctx, dwf_coarse and dwf_mg objects and their workspaces; the matching
 *   *_destroy call frees them.
 *
 * Errors.  Every call returns DWF_OK (0) or a negative status.  The library
 *   never exits, aborts or traps; dwf_last_error() describes the last failure
 *   of a context.  A CUDA error leaves the context usable only if the CUDA
 *   context itself is still usable.
 */
#ifndef DWFMG_H
#define DWFMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DWF_OK 0
#define DWF_EINVAL (-1)   /* bad argument: size, pointer, alignment, precision */
#define DWF_ENOMEM (-2)   /* device or host allocation failed */
#define DWF_ENOCONV (-3)  /* solver hit maxiter before the tolerance */
#define DWF_ENAN (-4)     /* NaN or Inf met in a solver or filter */
#define DWF_ECUDA (-5)    /* a CUDA runtime call failed */
#define DWF_ETIMEOUT (-6) /* a bounded device wait gave up */
#define DWF_ERANGE (-7)   /* filter overflow: the spectrum is not inside [lo, hi] */

#define DWF_F64 0
#define DWF_F32 1
#define DWF_F16S 2

#define DWF_EVEN 0
#define DWF_ODD 1

/* Solver precision policies for rbcg_solve. */
#define DWF_SOLVE_F64 0       /* every operation in FP64 */
#define DWF_SOLVE_MIXED_F32 1 /* FP32 inner CG, FP64 reliable updates */
#define DWF_SOLVE_MIXED_F16 2 /* FP16-storage inner CG, FP64 reliable updates */

typedef struct dwf_ctx dwf_ctx;
typedef struct dwf_coarse dwf_coarse;
typedef struct dwf_mg dwf_mg;

/* Statistics returned by the solvers.  "Matmuls" are counted in the paper's
 * unit: one full-lattice application of D_DW (or H_DW); a red-black CG
 * iteration (four half-lattice hopping terms) counts two (Sec. 5.1). */
typedef struct dwf_solve_stats {
  int iterations;            /* CG iterations, or outer GCR iterations (mg_solve) */
  int reliable_updates;      /* FP64 residual recomputations (mixed policies) */
  int coarse_iterations;     /* total coarse CG iterations (mg_solve) */
  int status;                /* same as the return value */
  double fine_matmuls;       /* full-lattice D_DW/H_DW applications, paper units */
  double true_residual;      /* ||b - D_DW x|| / ||b|| in FP64 at exit */
  double seconds;            /* wall time of the call (host clock) */
  double setup_seconds;      /* mg_setup phases: subspace filter */
  double coarse_op_seconds;  /* mg_setup phases: coarse operator build */
  int graph_replays;         /* mg_solve: V-cycles replayed from a CUDA graph;
                                rbcg_solve, rbcg2_solve, rbcg_normal_solve: blocks
                                of 8 CG iterations replayed from a CUDA graph */
  int pad_;
} dwf_solve_stats;

/* ------------------------------------------------------------------ context */

/* Create a context for an L[0]xL[1]xL[2]xL[3]xLs Shamir DWF operator with
 * domain-wall height M5 (Eq. 4-5; the paper leaves M5 open, the workloads use
 * 1.8).  `gauge` is the complex128 link field described above, host or
 * device; the context keeps parity-split copies of it in FP64, FP32 and FP16
 * (forward links U_mu(x) and backward links U_mu(x-mu)^dag stored side by
 * side per site).  Returns DWF_EINVAL for odd extents or unsupported Ls,
 * DWF_ENOMEM if the copies do not fit.  Synchronises `stream`. */
int dwf_ctx_create(dwf_ctx** ctx, const int L[4], int Ls, double M5,
                   const void* gauge, void* stream);
int dwf_ctx_destroy(dwf_ctx* ctx);
const char* dwf_last_error(const dwf_ctx* ctx);
/* Number of sites per parity (Vh) and the byte size of one half field of the
 * given precision, for allocation by the caller. */
int64_t dwf_half_sites(const dwf_ctx* ctx);
int64_t dwf_half_bytes(const dwf_ctx* ctx, int prec);

/* Kernel-launch and traffic counters of a context, for benchmarking:
 * *launches = kernels this library launched through the context since the
 * last reset; *hop_bytes = algorithmic (compulsory) bytes of the hopping-term
 * launches among them: per launch Vh*(Ls*nrhs*(24 [+12 with an aux input])
 * complex spinor numbers + 72 link complex numbers).  Host-side, no sync. */
int dwf_counters(const dwf_ctx* ctx, int64_t* launches, double* hop_bytes);
int dwf_reset_counters(dwf_ctx* ctx);

/* Autotuner of the hopping kernel: times every tuning variant (register cap x
 * inner-loop form: scalar, neighbour prefetch, packed FP32 on (re, im) pairs,
 * 2^4 hypercube tiles, two s-slices per thread with packed FP32 over the
 * pair (loads into registers, or staged in shared memory by cp.async with 2,
 * 4 or 8 neighbours in flight), CTAs of 2 or 4 y-rows, the scalar form
 * with an L2 prefetch of the rows a CTA a wave later reads first; DWF_HOP_VARIANTS
 * variants for FP32 and FP16
 * storage at Ls >= 16, one otherwise; for DWF_F64 the one FP64 kernel, or
 * with DWF_ARITH_FLOAT_FLOAT the float-float kernel under four register
 * caps) on this context's lattice, `reps`
 * launches each, keeps the fastest for precision `prec` and returns its time
 * per launch in *best_ms (may be NULL).  Variants that do not tile the
 * lattice are skipped.  Uses two half fields of context workspace, released
 * before returning; tuning launches are not counted.  Synchronises.  dwf_set_hop_variant / dwf_get_hop_variant pin or
 * read the choice (0 = untuned default; valid ids 0 .. DWF_HOP_VARIANTS-1;
 * dwf_set_hop_variant returns DWF_EINVAL for a variant that does not tile
 * the lattice). */
#define DWF_HOP_VARIANTS 26

/* Arithmetic of the FP64-precision hopping launches of a context (every
 * DWF_F64 D_hop, M_pc, D_DW and H_DW application, including the FP64
 * operator of the solvers: source preparation, reliable updates,
 * reconstruction, true residual).  DWF_ARITH_FP64 (default): FP64 units.
 * DWF_ARITH_FLOAT_FLOAT: the same FP64 fields computed on the FP32 units in
 * float-float arithmetic (pairs of FP32 numbers with error-free sums and
 * products, about 46 significant bits; Eq. 2 and Eq. 4 unchanged), several
 * times faster on GB300, whose FP64 rate is 1/74 of its FP32 rate.  FP64
 * inputs below 2^-126 in magnitude enter as zero.  The site-local kernel
 * and the BLAS stay FP64.  Host-side, no sync. */
#define DWF_ARITH_FP64 0
#define DWF_ARITH_FLOAT_FLOAT 1
int dwf_set_f64_arithmetic(dwf_ctx* ctx, int mode);
int dwf_get_f64_arithmetic(const dwf_ctx* ctx);
int dwf_autotune(dwf_ctx* ctx, int prec, int reps, double* best_ms, void* stream);
int dwf_set_hop_variant(dwf_ctx* ctx, int prec, int variant);
int dwf_get_hop_variant(const dwf_ctx* ctx, int prec);

/* ------------------------------------------------------------------ operators */

/* Wilson hopping term, Eq. (2), between parities: out (parity out_parity) =
 * D_hop in (parity 1-out_parity), applied on every s-slice with the same
 * links.  dagger=1 applies D_hop^dag (= gamma_5 D_hop gamma_5: the spin
 * projectors (1 -+ gamma_mu) swap).  nrhs half fields in, nrhs out. */
int dwf_dhop(dwf_ctx* ctx, void* out, const void* in, int out_parity, int dagger,
             int prec, int nrhs, void* stream);

/* Site-local part of D_DW, Eq. (4) without the hopping term of Eq. (5):
 * (M psi)_s = (5-M5) psi_s - P_- psi_{s+1} - P_+ psi_{s-1}, with mf P_+
 * psi_{Ls-1} at s = 0 and mf P_- psi_0 at s = Ls-1.  M_ee = M_oo = M.
 * dwf_mooee applies M (or M^dag), dwf_mooee_inv applies M^-1 (or M^-dag),
 * both on nrhs half fields; out may equal in. */
int dwf_mooee(dwf_ctx* ctx, void* out, const void* in, double mf, int dagger,
              int prec, int nrhs, void* stream);
int dwf_mooee_inv(dwf_ctx* ctx, void* out, const void* in, double mf, int dagger,
                  int prec, int nrhs, void* stream);

/* Red-black Schur operator of Sec. 5.1 (Table 5, first prec-CGNR row):
 * M_pc = M_ee - M_eo M_oo^-1 M_oe with M_eo = -1/2 D_hop(even<-odd).
 * dwf_mpc applies M_pc (or M_pc^dag) and dwf_mpcdag_mpc applies
 * M_pc^dag M_pc to nrhs even half fields.  Odd-parity temporaries come from
 * the context's workspace. */
int dwf_mpc(dwf_ctx* ctx, void* out, const void* in, double mf, int dagger,
            int prec, int nrhs, void* stream);
int dwf_mpcdag_mpc(dwf_ctx* ctx, void* out, const void* in, double mf, int prec,
                   int nrhs, void* stream);

/* Full-lattice D_DW (Eq. 4), its adjoint, and H_DW = Gamma_5 D_DW (Eq. 6,
 * Gamma_5 = gamma_5 R_5) on nrhs full fields. */
int dwf_ddw(dwf_ctx* ctx, void* out, const void* in, double mf, int dagger,
            int prec, int nrhs, void* stream);
int dwf_hdw(dwf_ctx* ctx, void* out, const void* in, double mf, int prec,
            int nrhs, void* stream);

/* ------------------------------------------------------------------ BLAS-1 */

/* Global reductions of the Krylov solvers (Sec. 5.1, Sec. 3.3) with FP64
 * accumulation over n complex numbers of the given precision: *result = sum |a|^2, or (re, im) of sum conj(a) b.
 * `result` is host memory; the call synchronises `stream`. */
int dwf_norm2(dwf_ctx* ctx, double* result, const void* a, int64_t n, int prec, void* stream);
int dwf_cdot(dwf_ctx* ctx, double* result2, const void* a, const void* b, int64_t n,
             int prec, void* stream);

/* Allocation-free |a|^2 (the paper has no counterpart; this serves callers
 * that cannot call cudaMalloc when they need a global sum, e.g. code running
 * under a memory pool that forbids new allocations or a plug-in handed only
 * its buffers).  |a|^2 of n complex numbers of precision prec at device address
 * a, summed in FP64 in a fixed order; *result on host.  For FP64 data this is
 * dwf_norm2's result up to summation order; for FP32 and FP16-storage data it
 * agrees with dwf_norm2 (which sums each thread's share in compensated FP32)
 * to within that FP32 reduction error (about 1e-7 relative).
 * Needs no context and allocates nothing: the reduction scratch is a static
 * device array in the library (512 KiB per GPU that loads it, held until
 * exit).  n <= 2^31, else DWF_EINVAL.  All calls on a device share that
 * scratch: calls that overlap on the GPU race.  The first call on a device
 * looks up the scratch address and should come before any stream capture;
 * the address is cached for the device's primary context, so the call must
 * not be used on a device again after cudaDeviceReset in the same process.
 * Returns DWF_ECUDA if a launch or the copy of the result fails.
 * Synchronises `stream`. */
int dwf_norm2_noalloc(double* result, const void* a, int64_t n, int prec, void* stream);

/* Self-test of the bounded device waits (no counterpart in the paper): runs
 * the two wait forms the kernels use -- polling a global counter and waiting
 * on an mbarrier phase -- against events that never happen, each limited to
 * about a millisecond.  gave_up[0] / gave_up[1] receive 1 when the poll / the
 * mbarrier wait gave up.  Returns DWF_ETIMEOUT when both gave up (the
 * expected outcome: the GPU stays usable and the status reaches the host),
 * DWF_OK if either wait unexpectedly completed.  Synchronises `stream`. */
int dwf_selftest_wait_timeout(int* gave_up, void* stream);

/* Measured fused multiply-add rates of this GPU's CUDA cores (no counterpart
 * in the paper: the ALU roof for the FP64 hopping kernel and the FP64 parts
 * of the solvers, measured instead of taken from a spec sheet).  Runs 8
 * independent FMA chains per thread on 8 CTAs of 256 threads per SM, best of
 * three timed launches per type (CUDA events); 2 flops per FMA.  Results in
 * TFLOP/s on the host.  Synchronises `stream`.  DWF_ECUDA if a launch fails. */
int dwf_measure_fma_peaks(double* fp64_tflops, double* fp32_tflops, void* stream);

/* ------------------------------------------------------------------ solvers */

/* Red-black preconditioned CGNR (Sec. 5.1): solve D_DW x = b for a full
 * field b (FP64, host or device), writing the full FP64 solution x (same
 * memory kind as b).  Prepares b'_e = b_e - M_eo M_oo^-1 b_o, runs CG on
 * M_pc^dag M_pc x_e = M_pc^dag b'_e and reconstructs x_o = M_oo^-1 (b_o -
 * M_oe x_e).  Stops when the FP64 true residual ||b - D_DW x|| / ||b|| <= tol
 * (returned in stats->true_residual), or returns DWF_ENOCONV after maxiter
 * CG iterations.  policy is one of DWF_SOLVE_*: with DWF_SOLVE_MIXED_F16 the
 * inner CG stores its vectors in FP16 (FP32 arithmetic) and works on the
 * residual scaled to unit mean square at every FP64 reliable update.  stats
 * may be NULL. */
int rbcg_solve(dwf_ctx* ctx, void* x, const void* b, double mf, double tol, int maxiter,
               int policy, dwf_solve_stats* stats, void* stream);

/* The second Schur form of Table 5 (second prec-CGNR row): the same
 * red-black solve of D_DW x = b with the even operator
 * M2 = 1 - M_ee^-1 M_eo M_oo^-1 M_oe = M_ee^-1 M_pc: CG on M2^dag M2 x_e =
 * M2^dag M_ee^-1 b'_e, then x_o = M_oo^-1 (b_o - M_oe x_e).  Same buffers,
 * stopping rule (FP64 true residual of D_DW), stats and errors as
 * rbcg_solve; policy DWF_SOLVE_F64 or DWF_SOLVE_MIXED_F32 (DWF_EINVAL
 * otherwise).  The paper's comparison point: more iterations than the first
 * form for the same residual. */
int rbcg2_solve(dwf_ctx* ctx, void* x, const void* b, double mf, double tol, int maxiter,
                int policy, dwf_solve_stats* stats, void* stream);

/* CG on the even normal equations M_pc^dag M_pc x = phi (Sec. 2.1, Eq. 9),
 * the pseudofermion solve of HMC: phi and x are FP64 even half fields in
 * device memory; stops when ||phi - M_pc^dag M_pc x|| / ||phi|| <= tol
 * (FP64, recomputed at every reliable update).  policy DWF_SOLVE_F64 or
 * DWF_SOLVE_MIXED_F32.  Synchronises. */
int rbcg_normal_solve(dwf_ctx* ctx, void* x, const void* phi, double mf, double tol, int maxiter,
                      int policy, dwf_solve_stats* stats, void* stream);

/* Unpreconditioned CGNR on the full lattice (the baseline row of the Krylov
 * comparison of Sec. 5.1: CG on D_DW^dag D_DW x = D_DW^dag b without the
 * red-black Schur complement), FP64 throughout.  x and b: full FP64 fields in
 * device memory (layout as for rbcg_solve, x must not alias b).  The
 * normal-equation residual is checked every 8 iterations; when it falls
 * below tol times |D_DW^dag b| the FP64 true residual ||b - D_DW x|| / ||b||
 * decides, and the normal-equation target tightens tenfold if it is above
 * tol.  stats: iterations, fine_matmuls (full-lattice D_DW or D_DW^dag
 * applications, two per iteration), true_residual.  DWF_ENOCONV after maxiter
 * iterations.  Synchronises. */
int cgnr_solve(dwf_ctx* ctx, void* x, const void* b, double mf, double tol, int maxiter,
               dwf_solve_stats* stats, void* stream);

/* Batched red-black CGNR (Sec. 5.1 operator; several pseudofermion masses on
 * one gauge field, as in the HMC of Sec. 6): solves D_DW(mf[i]) x_i = b_i for
 * i < nrhs (1 <= nrhs <= 64), each rhs with its own mass.  b and x hold nrhs
 * full FP64 fields back to back, each laid out as for rbcg_solve (even half,
 * then odd half); both host or both device, 16-byte aligned.  Each CG
 * iteration is one set of hopping launches over the systems still iterating
 * (the links are read once per launch for all of them); each system keeps its
 * own CG scalars and takes its own FP64 reliable updates, when the
 * single-system solver would.  A system whose FP64 true residual has reached
 * tol leaves the batch (its vectors are moved behind the active ones), so the
 * launches shrink as the heavier masses converge.  stats (NULL or nrhs
 * entries) receives per-system iterations (the iteration at which it reached
 * tol), reliable updates, fine matmuls, true residuals and status; seconds is
 * the wall time of the whole batch.  A zero source gives x_i = 0.  policy
 * DWF_SOLVE_F64 or DWF_SOLVE_MIXED_F32.  Returns DWF_ENOCONV if any system
 * missed tol after maxiter iterations (x is still written), DWF_EINVAL for
 * bad arguments or a non-finite mass.  Workspace: about 18 FP64 half fields
 * per system.  Synchronises. */
int rbcg_solve_batch(dwf_ctx* ctx, void* x, const void* b, const double* mf, int nrhs, double tol,
                     int maxiter, int policy, dwf_solve_stats* stats, void* stream);

/* Batched form of rbcg_normal_solve: M_pc(mf[i])^dag M_pc(mf[i]) x_i = phi_i
 * for i < nrhs, with phi and x nrhs FP64 even half fields back to back in
 * device memory (x must not alias phi).  Same batching, per-system reliable
 * updates, stats and errors as rbcg_solve_batch.  Synchronises. */
int rbcg_normal_solve_batch(dwf_ctx* ctx, void* x, const void* phi, const double* mf, int nrhs, double tol,
                            int maxiter, int policy, dwf_solve_stats* stats, void* stream);

/* Pseudofermion force (HMC context of Sec. 6; the paper prints no force, it
 * is derived for the Schur operator of Sec. 5.1): for each of npf even fields
 * X_i = (M_pc^dag M_pc)^-1 phi_i (mass mf[i], host array) this adds to
 * `force` (device complex128 [T][Z][Y][X][mu][3][3], the gauge layout)
 *   G_mu(x) = TA(U_mu(x) A_mu(x) - B_mu(x) U_mu(x)^dag),
 * A_mu(x) = sum_s tr_spin[(1-gamma_mu) X'_s(x+mu) Y'_s(x)^dag],
 * B_mu(x) = sum_s tr_spin[(1+gamma_mu) X'_s(x) Y'_s(x+mu)^dag],
 * with Y = M_pc X, X' = X + M_oo^-1 M_oe X, Y' = Y + M_oo^-dag M_eo^dag Y and
 * TA(M) = (M - M^dag)/2 - tr(M - M^dag)/6.  Convention: for U -> exp(eps Q) U
 * with Q in su(3), dS/deps = sum Re tr(G^dag Q) where S = sum_i phi_i^dag
 * (M_pc^dag M_pc)^-1 phi_i.  X: npf even half fields of precision prec (DWF_F64
 * or DWF_F32), device memory. */
int dwf_force(dwf_ctx* ctx, void* force, const void* X, const double* mf, int npf, int prec,
              void* stream);

/* Hasenbusch ratio factors (Sec. 6: the intermediate determinant ratios
 * det[M(m1)^dag M(m1)] / det[M(m2)^dag M(m2)] of the HMC), represented by
 *   S_r = phi^dag M2 (M1^dag M1)^-1 M2^dag phi,  M_i = M_pc(m_i)  (Sec. 5.1).
 * With X = (M1^dag M1)^-1 M2^dag phi (the caller's normal solve of
 * chi = M2^dag phi, e.g. rbcg_normal_solve after dwf_mpc with dagger = 1),
 * dS_r = 2 Re phi^dag dM2 X - 2 Re (M1 X)^dag dM1 X, and this call adds
 *   G_r = G(X', (M1 X)'; m1) - G(X', phi'; m2)
 * to `force` for each of nratio factors (1 <= nratio <= 32), G the bilinear
 * force of dwf_force with the full fields R' = R + M_oo^-1 M_oe R and
 * L' = L + M_oo^-dag M_eo^dag L at that term's mass.  Same convention,
 * layouts and force buffer as dwf_force; X and phi: nratio even half fields
 * of precision prec (DWF_F64 or DWF_F32) back to back, device memory;
 * m1, m2: host arrays of nratio finite masses.  With m1 = m2 the factor is
 * phi^dag phi and its force vanishes.  DWF_EINVAL for bad arguments,
 * DWF_ENOMEM when the workspace (eight half fields per factor) does not fit. */
int dwf_ratio_force(dwf_ctx* ctx, void* force, const void* X, const void* phi, const double* m1,
                    const double* m2, int nratio, int prec, void* stream);

/* Pseudofermion action by the variational estimator (HMC context of Sec. 6
 * on the operator of Sec. 5.1):
 *   *S = sum_i [2 Re <phi_i, X_i> - |M_pc(mf[i]) X_i|^2]
 * for npf FP64 even half fields phi, X back to back in device memory (X an
 * approximate (M_pc^dag M_pc)^-1 phi; the estimator's error is quadratic in
 * the solve's).  With phi replaced by chi = M2^dag phi and mf by m1 it is the
 * action of the ratio factors of dwf_ratio_force.  FP64 sums; *S on host;
 * DWF_ENAN if the result is not finite.  Synchronises. */
int dwf_pf_action(dwf_ctx* ctx, double* S, const void* phi, const void* X, const double* mf, int npf,
                  void* stream);

/* Power method estimate of the largest eigenvalue of D_DW^dag D_DW (Sec. 3.4),
 * `iters` iterations (v <- A v / |A v|, lambda = <v, A v>) from the FP64 full
 * field v0 (device), arithmetic in precision prec (DWF_F64 or DWF_F32: the
 * estimate only bounds a filter interval).  *lmax on host; synchronises. */
int dwf_power_max(dwf_ctx* ctx, double* lmax, const void* v0, double mf, int iters, int prec,
                  void* stream);

/* ------------------------------------------------------------------ subspace setup */

/* Chebyshev filter (Sec. 3.2, Eq. 23; Sec. 3.4, Eq. 34): out = T_order(x(A)) in
 * for nrhs full fields, A = D_DW^dag D_DW, x(A) = 2(A - lo)/(hi - lo) - 1, by
 * the three-term recurrence.  prec DWF_F64 or DWF_F32.  Returns DWF_ERANGE if
 * the result overflows (the spectrum of A reaches far beyond [lo, hi]). */
int cheby_filter(dwf_ctx* ctx, void* out, const void* in, int nrhs, double lo, double hi, int order,
                 double mf, int prec, void* stream);

/* Recursive subspace filter of Sec. 3.4 (Eqs. 34-37): phi_0 = T_m(2(A -
 * lam_lo)/(lam_max - lam_lo) - 1) eta, then phi_k = T_{k delta}(2A/lam_max - 1)
 * phi_0 for k = 1..nvec-1 as snapshots of one recurrence (cost m + (nvec-1)
 * delta applications of A).  eta is one full field, phi receives nvec full
 * fields, each normalised to unit norm.  Synchronises. */
int cheby_recursive_basis(dwf_ctx* ctx, void* phi, const void* eta, double lam_lo, double lam_max,
                          int m, int delta, int nvec, double mf, int prec, void* stream);

/* Chirality projection (Sec. 3.4, last paragraph): out = (1 + sign Gamma_5)/2
 * in on nrhs full fields, Gamma_5 = gamma_5 R_5; sign = +1 or -1; out may
 * equal in.  prec DWF_F64 or DWF_F32. */
int dwf_chiral_project(dwf_ctx* ctx, void* out, const void* in, int sign, int prec, int nrhs,
                       void* stream);

/* Block orthonormalisation of nb FP64 full fields in place so that P^dag P = 1
 * (implied by Sec. 3.1, Eq. 18): blocks are block[0..3] 4D sites times all of
 * Ls; vectors 0..nplus-1 and nplus..nb-1 (the two chiralities) are
 * orthonormalised separately, in index order, by Cholesky-QR applied twice
 * (the same Q as modified Gram-Schmidt in exact arithmetic).  Groups of at
 * most 32 vectors.  DWF_ERANGE if the vectors are dependent on a block. */
int block_orthonormalise(dwf_ctx* ctx, void* basis, int nb, int nplus, const int block[4],
                         void* stream);

/* ------------------------------------------------------------------ coarse operator */

/* Little Dirac operator of H_DW (Sec. 3.1, Eq. 18; Table 1 "Coarsening H_DW"):
 * A_d(x)_{jk} = <phi^x_j, H^(d) phi^{x+d}_k> for the 9 stencil directions d =
 * 0 (self), +x, -x, +y, -y, +z, -z, +t, -t, on the coarse lattice L/block.
 * basis: nb orthonormal block vectors as full fields of precision prec
 * (DWF_F64 or DWF_F32); vectors 0..nplus-1 have Gamma_5 = +1.  The library
 * owns the result (FP64 and FP32 copies). */
int coarse_build(dwf_ctx* ctx, const void* basis, int nb, int nplus, const int block[4], double mf,
                 int prec, dwf_coarse** coarse, void* stream);
int coarse_destroy(dwf_coarse* coarse);
/* Copy the FP64 operator of Eq. (18) (Sec. 3.1) to A (host or device,
 * complex128 [nc][9][nb][nb], row j, column k) and/or its shape to dims = {Lc_x, Lc_y, Lc_z, Lc_t, nb}. */
int coarse_export(const dwf_coarse* coarse, void* A, int* dims);
/* The 9-point stencil of Eq. (18) (Sec. 3.1) on nrhs coarse vectors:
 * out(x) = sum_d A_d(x) in(x+d), FP32 complex, layout
 * [nc][nb][nrhs] (coarse site lexicographic in Lc, basis index, rhs).
 * prec DWF_F32: CUDA cores, FP32 arithmetic (any nb, nrhs).  prec DWF_TF32:
 * 5th-generation tensor cores (tcgen05.mma kind::tf32, inputs rounded to TF32,
 * FP32 accumulation in tensor memory) for nb = 32, an even number of coarse
 * sites and nrhs in {16, 32, 64}; other shapes return DWF_EINVAL.  Both
 * paths are asynchronous on `stream`.  The tensor-core kernel's waits are
 * bounded: one that gives up raises a sticky flag of the operator, which a
 * later TF32 coarse_apply returns as DWF_ETIMEOUT once its copy to the host
 * has landed, and coarse_apply_status returns after synchronising. */
#define DWF_TF32 3
int coarse_apply(dwf_coarse* coarse, void* out, const void* in, int nrhs, int prec, void* stream);
/* Synchronise `stream` and return DWF_ETIMEOUT if a bounded wait of an
 * earlier tensor-core coarse_apply on this operator gave up (the flag is then
 * cleared), else DWF_OK. */
int coarse_apply_status(dwf_coarse* coarse, void* stream);
/* Coarse solve of Table 1 ("Coarse solver: CGNR"): CG on A^2 e = A r for one
 * FP32 coarse vector, stopping when the normal residual is below tol times its
 * initial value or after maxiter iterations (*iters receives the count). */
int coarse_solve(dwf_coarse* coarse, void* e, const void* r, double tol, int maxiter, int* iters,
                 void* stream);
/* Coarse solves for many right-hand sides (the multi-RHS use of the little
 * Dirac operator, Sec. 3.1): CG on A^2 e_r = A rhs_r for nrhs independent
 * FP32 right-hand sides at once (layout [nc][nb][nrhs], e the same), each
 * with its own step lengths and FP64 scalars; every application of A covers
 * all of them, on the tensor cores (prec DWF_TF32, the shapes coarse_apply
 * accepts: nb = 32, nrhs 16 or 32 or 64) or on the CUDA cores (DWF_F32,
 * nrhs dividing 256).  A right-hand side stops changing once its normal
 * residual |A^2 e_r - A rhs_r| <= tol |A rhs_r| (checked every 8 iterations);
 * iters (host, nrhs entries, may be NULL) receives the iteration at which each
 * did.  The TF32 operator carries a relative error of about 5e-4, so tol
 * below about 1e-3 is not reached with DWF_TF32 (DWF_ENOCONV after maxiter).
 * Synchronises. */
int coarse_solve_multi(dwf_coarse* coarse, void* e, const void* rhs, int nrhs, double tol, int maxiter,
                       int* iters, int prec, void* stream);
/* Red-black coarse solve (Sec. 5.3: the red-black coarse solver of the
 * physical-point runs): with even coarse extents the 9-point stencil couples
 * a coarse site only to itself and to the other coarse parity, so A e = r is
 * solved by CG on S^2 e_e = S r'_e with the even Schur complement
 * S = A_ee - A_eo A_oo^-1 A_oe (hermitian; A_oo^-1 = the nb x nb self-block
 * inverses), r'_e = r_e - A_eo A_oo^-1 r_o, then e_o = A_oo^-1 (r_o - A_oe
 * e_e).  Stops when |S^2 e_e - S r'_e| <= tol |S r'_e| or after maxiter
 * iterations (*iters).  Parity of a coarse site: (xc + yc + zc + tc) mod 2.
 * The first call inverts the odd self blocks in FP64 (Gauss-Jordan with
 * partial pivoting) and keeps A_oo^-1 and A_oo^-1 A_oe with the operator
 * (FP32, the size of the operator).  FP32 vectors [nc][nb].  DWF_EINVAL for
 * odd coarse extents or nb > 64, DWF_ERANGE for a singular self block.
 * Synchronises. */
int coarse_solve_rb(dwf_coarse* coarse, void* e, const void* r, double tol, int maxiter, int* iters,
                    void* stream);
/* Coarse-space deflation (Sec. 3.5: eigenvector deflation of the coarse
 * operator with Chebyshev-polynomial-preconditioned Lanczos).  Lanczos with
 * full reorthogonalisation runs nk steps on B = T_order(y(A^2)),
 * y(t) = 2 (t - lam_lo) / (lam_max - lam_lo) - 1 (order even, >= 2), from the
 * caller's start vector v0 (FP32 coarse vector [nc][nb], device); the nev
 * Ritz vectors of B's largest Ritz values are then diagonalised with A^2
 * (Rayleigh-Ritz), giving pairs (theta_i, v_i), theta ascending, written to
 * theta (host, may be NULL).  lam_max <= 0: a 30-step power method on A^2
 * (+10 %) sets it.  The operator keeps the v_i (nev FP32 coarse vectors) and
 * from then on coarse_solve -- and the multigrid's plain coarse CG -- start
 * from x0 = sum_i v_i <v_i, A r> / theta_i, with the stopping rule still
 * relative to the residual of the zero start.  nev = 0 drops the space.
 * Needs 1 <= nev <= nk <= min(1024, nc nb); DWF_EINVAL otherwise,
 * DWF_ERANGE if the Krylov space closes before nev vectors or a Ritz value
 * is not positive.  Small dense eigenproblems on the host (Jacobi).
 * Synchronises. */
int coarse_deflate(dwf_coarse* coarse, const void* v0, int nev, int nk, int order, double lam_lo,
                   double lam_max, double* theta, void* stream);
/* The coarse deflation space of Sec. 3.5 (coarse_deflate): *nev vectors (FP32 [nev][nc][nb],
 * copied to V, host or device, when V is not NULL) and 1/theta_i (host). */
int coarse_export_deflation(const dwf_coarse* coarse, void* V, double* theta_inv, int* nev);
/* Restriction P^dag (out: FP32 coarse [nc][nb][nrhs]) and prolongation P
 * (out: nrhs full fields, += when accumulate) with a block basis of nb full
 * fields of precision prec (DWF_F64 or DWF_F32): the block projectors of
 * Sec. 3.1 that Eqs. (26)-(28) use. */
int dwf_restrict(dwf_ctx* ctx, void* out, const void* in, const void* basis, int nb,
                 const int block[4], int nrhs, int prec, void* stream);
int dwf_prolong(dwf_ctx* ctx, void* out, const void* in, const void* basis, int nb,
                const int block[4], int nrhs, int prec, int accumulate, void* stream);

/* ------------------------------------------------------------------ HDCR multigrid */

#define DWF_SUBSPACE_BATCH 0     /* nbasis Gaussians filtered together by T_order */
#define DWF_SUBSPACE_RECURSIVE 1 /* nbasis/2 vectors from one Gaussian (Sec. 3.4) */

/* Parameters of Table 1 (Algorithms A, B) and Table 12 (Algorithm H). */
typedef struct dwf_mg_params {
  int block[4];          /* 4D block; the block spans all of Ls */
  int nbasis;            /* basis vectors after chirality projection (even, <= 64) */
  int subspace_mode;     /* DWF_SUBSPACE_* */
  double mf;             /* quark mass of D_DW */
  double lambda_lo;      /* subspace lambda_lo */
  double lambda_max;     /* subspace lambda_max (must bound spec(D^dag D)) */
  int filter_order;      /* m (recursive) or the batch filter order */
  int delta;             /* Delta of the recursive filter */
  double smooth_lo;      /* smoother interval [a, b] of S_cheb([a,b],N) on H_DW^2 */
  double smooth_hi;
  int smooth_order;      /* N */
  double coarse_tol;     /* coarse CG relative tolerance (0.02 in Table 12) */
  int coarse_maxiter;
  int nkrylov;           /* GCR restart length */
  int maxiter;           /* outer iterations */
  int no_graph;          /* 0: mg_solve captures the V-cycle in a CUDA graph
                            once per solve and replays it; 1: plain launches */
  int coarse_solver;     /* DWF_COARSE_CG: CG on A^2 (Table 1); DWF_COARSE_RB:
                            red-black CG on S^2 (coarse_solve_rb, Sec. 5.3);
                            DWF_COARSE_DEFLATED: CG on A^2 started from the
                            deflation guess (coarse_deflate, Sec. 3.5), the
                            space built by mg_setup from the restriction of the
                            first eta */
  int coarse_nev;        /* deflation: Ritz vectors kept */
  int coarse_lanczos;    /* deflation: Lanczos steps */
  int coarse_cheb_order; /* deflation: even Chebyshev order of the Lanczos operator */
  double coarse_cheb_lo; /* deflation: modes of A^2 below this are enhanced */
} dwf_mg_params;

#define DWF_COARSE_CG 0
#define DWF_COARSE_RB 1
#define DWF_COARSE_DEFLATED 2

/* Build the multigrid setup: filtered vectors from eta (nbasis FP64 full fields
 * in batch mode, one in recursive mode; device memory), chirality projection
 * ((1+Gamma_5)/2 for the first nbasis/2, (1-Gamma_5)/2 for the rest), FP64
 * block orthonormalisation, FP32 basis storage and the little Dirac operator
 * of H_DW.  Synchronises.  The context must outlive the setup. */
int mg_setup(dwf_ctx* ctx, const dwf_mg_params* params, const void* eta, dwf_mg** mg, void* stream);
int mg_destroy(dwf_mg* mg);
/* Copy the FP32 basis (nbasis full fields; Sec. 3.4) to out (host or device). */
int mg_export_basis(const dwf_mg* mg, void* out);
/* The setup's coarse operator (owned by the setup); for a hybrid setup
 * (mg_setup_hybrid) the level-2 operator. */
dwf_coarse* mg_coarse(dwf_mg* mg);
/* The Chebyshev smoother S_cheb (Sec. 3.2, Eqs. 24-25, with M = M^dag = H_DW)
 * and the V(1,1) preconditioner (Sec. 3.3, Eqs. 26-28, x0 = 0) applied to one
 * FP32 full field.  Synchronise. */
int mg_smooth(dwf_mg* mg, void* out, const void* in, void* stream);
int mg_precondition(dwf_mg* mg, void* out, const void* in, void* stream);
/* HDCR solve of D_DW x = b (Table 1: outer pGCR(H_DW)): flexible GCR on
 * H_DW x = Gamma_5 b preconditioned by V(1,1), FP64 x and true residual, FP32
 * directions; stops when ||b - D_DW x|| / ||b|| <= tol.  b, x: FP64 full
 * fields, host or device.  stats->fine_matmuls counts H_DW applications. */
int mg_solve(dwf_mg* mg, void* x, const void* b, double tol, dwf_solve_stats* stats, void* stream);

/* ------------------------------------------------------------------ hybrid three-level multigrid */

/* Algorithm F (Sec. 4 and its table; Hybrid-M^dag M): the first coarsening
 * represents the 4D Wilson operator D_W (Eq. 1) on 4D blocks with the fifth
 * dimension kept (blocks b^4 x 1); by the chirality of the 4D basis the level-1
 * operator is a coarse domain wall operator
 *   M_1 v(x,k,s) = sum_s' K_chi_k[s,s'] v(x,k,s') + sum_d sum_k' B_d(x)[k,k'] v(x+d,k',s),
 * K_chi the Ls x Ls fifth-dimension matrix of Eq. (4) on chirality chi_k (+1
 * for k < nbasis4/2) and B = P4^dag (-1/2 D_hop) P4 the 9-point stencil of the
 * hopping term on the 4D basis.  The second coarsening represents
 * H_1 = Gamma5_1 M_1 (Gamma5_1 v(x,k,s) = chi_k v(x,k,Ls-1-s)) on blocks of one
 * level-1 site spanning all s, a 9-point stencil with nbasis1 x nbasis1
 * blocks solved like the HDCR coarse operator (dwf_mg_params' coarse_*).
 * The fine outer solve is that of mg_solve; its V(1,1) coarse correction is
 * P1 e, e from kcycle iterations of flexible GCR on H_1 e = P1^dag r (no
 * tolerance test: a fixed W-cycle), each iteration preconditioned by a
 * level-1 V(1,1) whose coarse-coarse correction is the level-2 solve.
 *
 * Level-1 vectors: FP32 complex [nc1][nbasis4][Ls][nvec] (coarse site of the
 * 4D blocking, 4D basis index, s, vector), nc1 = prod(L/block).  Level-2
 * vectors: FP32 complex [nc1][nbasis1]. */
typedef struct dwf_hybrid_params {
  int block[4];          /* 4D blocks of the D_W coarsening (Algorithm F: 2^4) */
  int nbasis4;           /* 4D basis vectors: 4, 8, 16 or 24 (half of each chirality) */
  double mass4;          /* Wilson mass m of the filter operator D_W(m)^dag D_W(m), > -4 */
  double lambda_lo4;     /* batch filter T_order4 on [lambda_lo4, lambda_max4] */
  double lambda_max4;
  int order4;
  int nbasis1;           /* level-2 basis vectors (even, <= 64; half of each Gamma5_1 chirality) */
  double lambda_lo1;     /* batch filter T_order1 of H_1^2 on [lambda_lo1, lambda_max1] */
  double lambda_max1;
  int order1;
  double smooth1_lo;     /* level-1 smoother S_cheb([lo,hi],N) on H_1 (N = 0: none, */
  double smooth1_hi;     /*   only with kcycle = 1: without a smoother the level-1 */
  int smooth1_order;     /*   preconditioner K obeys K H_1 K = K) */
  int kcycle;            /* GCR iterations of the level-1 solve (2: the W-cycle) */
} dwf_hybrid_params;

/* Build the three levels: eta4 = nbasis4 Gaussian 4D fields (FP64, the layout
 * of a full field with Ls = nbasis4: [parity][Vh][4][3][nbasis4], vector
 * innermost), filtered in FP32 by T_order4 of D_W^dag D_W, projected with
 * (1 +- gamma_5)/2 (first half +), block orthonormalised and the stencil B
 * built in FP64; eta1 = nbasis1 Gaussian level-1 vectors (FP64
 * [nc1][nbasis4][Ls][nbasis1]) filtered in FP32 by T_order1 of H_1^2,
 * projected with (1 +- Gamma5_1)/2, orthonormalised per level-1 site (FP64
 * arithmetic, FP32 storage), and the level-2 stencil built (FP64 sums).
 * params supplies mf, the fine smoother, nkrylov, maxiter and the coarse
 * (level-2) solver and its deflation; its block, nbasis and subspace fields
 * are not used.  The solve runs without CUDA-graph replay.  Synchronises. */
int mg_setup_hybrid(dwf_ctx* ctx, const dwf_mg_params* params, const dwf_hybrid_params* hybrid,
                    const void* eta4, const void* eta1, dwf_mg** mg, void* stream);
/* Copies of the hybrid setup's parts (Algorithm F, Sec. 4; host or device out):
 *   what 0: the 4D basis, FP64 [2][Vh][12][nbasis4];
 *   what 1: B, FP64 [nc1][9][nbasis4][nbasis4] (the coarse_export layout);
 *   what 2: the level-2 basis, FP32 [nc1][nbasis4][Ls][nbasis1];
 *   what 3: the level-2 stencil, FP64 [nc1][9][nbasis1][nbasis1].
 * DWF_EINVAL for a setup that is not hybrid. */
int mg_hybrid_export(const dwf_mg* mg, int what, void* out);
/* The hybrid setup's level operators (Algorithm F, Sec. 4) on device vectors
 * (stream-ordered):
 *   op 0: out = M_1 in, nvec level-1 vectors;  op 1: out = H_1 in;
 *   op 2: out = P1^dag in (in: nvec FP32 full fine fields; out: level-1);
 *   op 3: out = P1 in (in: level-1; out: nvec FP32 full fields);
 *   op 4: out = P2^dag in (nvec = 1; out: level-2 vector);
 *   op 5: out = P2 in (nvec = 1; in: level-2 vector);
 *   op 6: out = the fixed-iteration level-1 solve of H_1 out = in (nvec = 1;
 *         synchronises).
 * out must not alias in. */
int mg_hybrid_level1(dwf_mg* mg, int op, void* out, const void* in, int nvec, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DWFMG_H */
