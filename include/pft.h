/*
 * pft.h -- C ABI of the GB300 partial Fourier transform (PFT) and PIE library.
 *
 * The library implements, on one GPU (sm_103a):
 *   - the 2-D fast partial Fourier transform of Parada, Wu Fung and Osher,
 *     "Fast Partial Fourier Transforms for Large-Scale Ptychography"
 *     (offline phase: Algorithm 4; online phase: Algorithm 5), which returns
 *     the lowest M x M Fourier coefficients of each n x n frame, and its exact
 *     adjoint;
 *   - the exact partial DFT (the Appendix-A 2-D DFT restricted to the lowest
 *     M x M frequencies) and a full 2-D FFT, for the refine phase and as
 *     baselines;
 *   - the PIE sweep (Section 2.1, Eq. pie_update with the modulus projection
 *     of Eq. 3), run with either the PFT or the full FFT, and the hybrid
 *     warm start of Algorithm 3;
 *   - the gradient of the amplitude loss through the PFT with respect to the
 *     object and the probe.
 *
 * Conventions (every call):
 *   - Complex arrays are interleaved single precision (real, imaginary),
 *     8 bytes per element, row-major. Real arrays are float.
 *   - "device" pointers are CUDA device memory owned by the caller; "host"
 *     pointers are ordinary host memory owned by the caller. The library never
 *     frees caller memory. Plans and contexts are opaque, owned by the library,
 *     and hold the tables, schedules and workspace they allocate.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Calls that take a stream enqueue work on it and return without
 *     synchronising unless documented otherwise.
 *   - The transform is unnormalised and uses e^{-2 pi i t k / n}. Output
 *     frequencies are centred: row index t1 + M1/2, column t2 + M2/2, with
 *     t in [-M/2, M/2 - 1]. The adjoint is the exact conjugate transpose of the
 *     operator the plan applies (unscaled).
 *   - Every call returns an int status: PFT_OK (0) or a negative PFT_ERR_*.
 *     On error outputs are unspecified; pft_last_error() returns a
 *     thread-local message. No C++ exception crosses the ABI.
 */
#ifndef PFT_GB300_H
#define PFT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PFT_OK                0
#define PFT_ERR_INVALID_ARG  (-1)  /* null pointer, bad size, bad enum           */
#define PFT_ERR_UNSUPPORTED  (-2)  /* valid request outside the built kernels    */
#define PFT_ERR_CUDA         (-3)  /* a CUDA runtime call failed                  */
#define PFT_ERR_NONFINITE    (-4)  /* NaN or Inf met in data or a result norm     */
#define PFT_ERR_TIMEOUT      (-5)  /* a device-side wait gave up (status word)    */
#define PFT_ERR_OOM          (-6)  /* device or host allocation failed            */

/* ---- enums ------------------------------------------------------------- */
#define PFT_PATH_AUTO        0   /* choose the factorised PFT when supported     */
#define PFT_PATH_FACTORISED  1   /* Algorithm 5 (polynomial factorisation)       */
#define PFT_PATH_DIRECT      2   /* exact partial DFT (dense M x n per axis)     */

#define PFT_PREC_FP32        0   /* FP32 CUDA-core arithmetic, FP32 accumulation */
#define PFT_PREC_SPLIT_BF16  1   /* tensor cores: BF16 hi + lo operand splits,
                                    three products per term, FP32 accumulation */

#define PIE_TRANSFORM_PFT    0   /* PIE with the plan's partial transform (M x M) */
#define PIE_TRANSFORM_FULL   1   /* PIE with the full n x n FFT                   */

#define PIE_MODE_COLOURED    0   /* sequential PIE, positions grouped in colours
                                    of non-overlapping patches (exact PIE order) */
#define PIE_MODE_BATCHED     1   /* all positions read the same object; updates
                                    summed and divided by the illumination       */

/* Launch forms of a coloured sweep (pie_ctx_set_persistent); all three give
 * the same result, bit for bit. */
#define PIE_LAUNCH_PER_COLOUR 0  /* one launch per colour                        */
#define PIE_LAUNCH_PERSISTENT 1  /* one cooperative launch, grid barrier between
                                    colours                                      */
#define PIE_LAUNCH_DATAFLOW   2  /* one cooperative launch over the colour-major
                                    schedule; a position waits only for the
                                    earlier positions whose patches overlap its
                                    own (no barrier between colours)             */

/* Probe step of a blind sweep (pie_iteration_blind). */
#define PIE_PROBE_STEP_NORMALISED 0  /* gamma sum_j g_j / (sum_j |z_j|^2 + delta),
                                        pixel by pixel, once per colour         */
#define PIE_PROBE_STEP_SCALAR     1  /* gamma sum_j g_j: Eq. epie_probe_update's
                                        plain scalar step                       */

/* Last error message of the calling thread ("" if none). Never NULL. */
const char* pft_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int pft_version(void);

/* ---- offline phase (host only, no GPU needed) ---------------------------
 * Section 3.1.1: best uniform approximation P_{r-1, xi}(x) = sum_j w_j x^j of
 * e^{i pi x} on |x| <= xi, with the scope xi(eps, r) = sup{xi : error <= eps}.
 * By symmetry w_j = i^j a_j with a_j real.
 *
 * pft_design_coefficients: for (eps, r) writes xi(eps, r) to *xi and the r
 *   real values a_0..a_{r-1} to a[] (host array of length >= r), and the
 *   uniform error of the polynomial on |x| <= xi to *err (may be NULL).
 *   1 <= r <= 32, 0 < eps < 1. Thread-safe; results are cached.
 * pft_choose_r: the choice of r in Algorithm 1, r = min{ r : xi(eps, r) >= ratio },
 *   ratio = m~/p = M/(2p). Writes r to *r (INVALID_ARG if none <= 32).
 */
int pft_design_coefficients(double eps, int r, double* xi, double* a, double* err);
int pft_choose_r(double eps, double ratio, int* r);

/* ---- plans (Algorithm 4) --------------------------------------------------
 * A plan fixes the frame size n1 x n2, the output size M1 x M2 and the
 * factorisation n_nu = p_nu q_nu. It computes the coefficients on the host
 * and the tables B_nu (q_nu x r_nu, real after taking i^j into W), W_nu
 * (M_nu x r_nu) and the DFT twiddles on the GPU in FP64 with exact integer
 * phase reduction, stored as FP32.
 *
 * pft_plan_create(out, n1, n2, M1, M2, p1, p2, eps, r1, r2, path, precision)
 *   n_nu: frame sides; M_nu: output sides (even, M_nu <= n_nu);
 *   p_nu: divisors of n_nu, 0 = auto (p = M/2, so m~/p = 1 as in Section 4);
 *   eps: polynomial tolerance (Section 4 uses 1e-7); r_nu: 0 = Algorithm 1's
 *   choice, else forced; path: PFT_PATH_*; precision: PFT_PREC_*.
 *   Synchronises the device once (table generation). UNSUPPORTED when the
 *   sizes are outside the built kernels (the message says which).
 * Built shapes (square frames, p = M/2):
 *   PFT_PREC_FP32        (n, M) in {(32, 16), (64, 16), (64, 32), (64, 64),
 *                        (128, 16), (128, 32), (128, 64), (256, 16),
 *                        (256, 32), (256, 64)} (forward and adjoint, CUDA
 *                        cores);
 *   PFT_PREC_SPLIT_BF16  n = 256 with M = 32 or M = 64 (forward and
 *                        adjoint), tensor cores with the per-axis operator
 *                        folded into one table (at M = 64 only the rows
 *                        t >= 0 and t = -M/2, using A[-t] = conj(A[t]));
 *                        n in {2048, 4096, 8192, 16384} with M = 128
 *                        (p = 64, q = n / 64; forward and adjoint): the
 *                        paper's large-frame regime, stage A of Algorithm 5
 *                        on tensor cores, stage B on CUDA cores; frames go in
 *                        passes through a plan-owned workspace of <= 32 MB.
 *   A split-BF16 plan's results carry a relative error of about 1e-5 per
 *   frame (BF16 hi + lo operands, three partial products per term).
 *   Device-side waits of the tensor-core kernels are bounded (2 s); a timeout
 *   is latched in the plan and returned as PFT_ERR_TIMEOUT by its next
 *   pft_forward / pft_adjoint call.
 */
typedef struct pft_plan pft_plan;

typedef struct pft_plan_info {
  int n1, n2, M1, M2;
  int p1, p2, q1, q2, r1, r2;   /* factorisation and polynomial terms per axis */
  double xi1, xi2;              /* scopes xi(eps, r_nu)                        */
  double eps;
  int path;                     /* PFT_PATH_FACTORISED or PFT_PATH_DIRECT      */
  int precision;
} pft_plan_info;

int pft_plan_create(pft_plan** out, int n1, int n2, int M1, int M2, int p1, int p2,
                    double eps, int r1, int r2, int path, int precision);
int pft_plan_destroy(pft_plan* plan);
int pft_plan_info_get(const pft_plan* plan, pft_plan_info* info);

/* Copy the plan's FP32 tables to host memory (for inspection and tests).
 * axis 0 or 1. B: q x r real (row-major, may be NULL); W: M x r complex
 * (row-major, includes the factor i^j, may be NULL). */
int pft_plan_tables(const pft_plan* plan, int axis, float* B, float* W);

/* ---- online phase: batched transforms ------------------------------------
 * pft_forward (Algorithm 5): x = device [batch][n1][n2] complex,
 *   y = device [batch][M1][M2] complex (centred). x and y must not overlap.
 * pft_adjoint: y = device [batch][M1][M2] -> x = device [batch][n1][n2],
 *   x = A^H y for the plan's operator A (unscaled).
 * batch >= 0 (0 is a no-op). Asynchronous on `stream`.
 */
int pft_forward(const pft_plan* plan, const void* x, void* y, int64_t batch, void* stream);
int pft_adjoint(const pft_plan* plan, const void* y, void* x, int64_t batch, void* stream);

/* ---- full FFT (baseline and refine phase) ---------------------------------
 * pft_fft2: unnormalised full 2-D DFT of n x n frames (inverse = 0) or its
 *   conjugate transpose (inverse = 1, i.e. n^2 times the inverse DFT);
 *   in/out device [batch][n][n], may alias. n in {16, 32, 64, 128}.
 * pft_fft_crop: full 2-D FFT of each n x n frame followed by the centred
 *   M x M crop (the naive route the PFT avoids); out device [batch][M][M].
 */
int pft_fft2(const void* in, void* out, int n, int64_t batch, int inverse, void* stream);
int pft_fft_crop(const void* in, void* out, int n, int M, int64_t batch, void* stream);

/* ---- PIE ------------------------------------------------------------------
 * A context holds one reconstruction problem: object size, probe, scan
 * positions, measured intensities and the plans it needs.
 *
 * pie_ctx_create(out, problem, probe, positions, intensities, stream)
 *   probe:       device [n][n] complex (copied; later changes to the caller's
 *                buffer are not seen);
 *   positions:   host int32 [N][2], top-left (row, col) of each n x n patch,
 *                0 <= row <= obj_h - n, 0 <= col <= obj_w - n;
 *   intensities: device float [N][n][n], far-field intensities in FFT order
 *                (not shifted). The context stores d = sqrt(I) and the
 *                centred crop d^crop (the cropped data of Algorithm 3);
 *                negative counts are taken as 0, and a NaN or infinite
 *                intensity makes the call return PFT_ERR_NONFINITE.
 *   Synchronises `stream`. The caller's buffers may be freed afterwards.
 */
typedef struct pie_ctx pie_ctx;

typedef struct pie_problem {
  int obj_h, obj_w;      /* object size                                       */
  int n;                 /* probe / frame side                                 */
  int npos;              /* N, number of scan positions                        */
  int M;                 /* PFT output side (even, <= n)                       */
  int p;                 /* PFT divisor (0 = auto, M/2)                        */
  double eps;            /* PFT polynomial tolerance (0 = 1e-7)                */
  int mode;              /* PIE_MODE_*                                         */
  int path;              /* PFT_PATH_* for the partial transform               */
  double delta_rel;      /* batched mode: delta = delta_rel * max illumination */
  int autotune;          /* 1: time every built kernel variant (CTAs per position)
                            on a scratch object at creation and keep the fastest;
                            in coloured mode also the same kernel run as one
                            cooperative launch per sweep (a grid barrier between
                            colours, bounded at 2 s: a timeout is returned as
                            PFT_ERR_TIMEOUT by the next pie_iteration);
                            0: pick by occupancy, one launch per colour           */
} pie_problem;

typedef struct pie_stats {
  double phi;            /* (1/N) sum_j ||R_j||^2 / n^2 during the sweep (Eq. 4) */
  double rel_change;     /* ||z_new - z_old|| / ||z_old||  (Section 4)           */
} pie_stats;

int pie_ctx_create(pie_ctx** out, const pie_problem* problem, const void* probe,
                   const int32_t* positions, const float* intensities, void* stream);
int pie_ctx_destroy(pie_ctx* ctx);

/* What the context chose: colours, PFT factorisation, and the CTAs per
 * position of the PFT and full-FFT sweeps picked by the autotuner (0 when not
 * tuned: chosen per launch by occupancy) with the sweep time it measured. */
typedef struct pie_ctx_info {
  int ncolours;
  int p, q, r;
  int cluster_pft, cluster_full;
  double sweep_ms_pft, sweep_ms_full;
  int persistent_pft, persistent_full;  /* launch form of the coloured sweeps:
                                           PIE_LAUNCH_* (the dataflow form
                                           reports its own cluster size above) */
} pie_ctx_info;

int pie_ctx_info_get(const pie_ctx* ctx, pie_ctx_info* info);

/* Number of colours of the greedy colouring (positions in index order take
 * the smallest colour unused by an earlier overlapping patch), and the
 * colour of each position (host int32 [N], may be NULL). */
int pie_ctx_colours(const pie_ctx* ctx, int* ncolours, int32_t* colour_of);

/* Host only (no GPU work, no allocation on the device): the order in which a
 * context with these positions sweeps them. The paper visits positions
 * sequentially (Section 2.1, Eq. pie_update); any visiting order is a valid
 * PIE order, and the library runs the positions colour by colour:
 *   colour   host int32 [npos]: greedy colouring in visiting order (each
 *            position takes the smallest colour unused by an earlier visited
 *            position whose patch overlaps its own; patches overlap when both
 *            corner coordinates differ by less than n);
 *   sched    host int32 [npos]: the colour-major schedule, visiting order
 *            within a colour (what every coloured sweep runs);
 *   dep_off  host int32 [npos + 1], dep host int32 [dep_capacity]: the
 *            predecessors of schedule item s (schedule indices
 *            dep[dep_off[s] .. dep_off[s + 1])) that the dataflow launch form
 *            waits for: the earlier items whose patches overlap item s, minus
 *            those that are also earlier overlapping items of another member
 *            of that set (waiting for the later one covers them).
 * positions: host int32 [npos][2] top-left (row, col), each patch inside the
 * obj_h x obj_w object; order: host int32 [npos] permutation or NULL (index
 * order); one_per_colour != 0: every position is its own colour, colour a
 * being the a-th position visited (the schedule is then the visiting order
 * itself). *ncolours and *ndep (the number of dep entries) are always written;
 * every other output may be NULL. INVALID_ARG for a patch outside the object,
 * an order that is not a permutation, or dep_capacity < *ndep with dep set. */
int pie_scan_schedule(const int32_t* positions, int npos, int n, int obj_h, int obj_w, const int32_t* order,
                      int one_per_colour, int* ncolours, int32_t* colour, int32_t* sched, int32_t* dep_off, int32_t* dep,
                      int64_t dep_capacity, int64_t* ndep);

/* One PIE sweep over all positions (Eq. pie_update with Eq. 3), in place on
 * `object` (device [obj_h][obj_w] complex). transform: PIE_TRANSFORM_*.
 * Step: beta * conj(w) / max|w|^2 (coloured) or
 * beta * conj(w) / (illumination + delta) (batched). For the PFT the
 * residual step is A^H(A psi - d^crop sgn(A psi)) / n^2.
 * If `stats` is non-NULL the call synchronises `stream` and fills it
 * (FP64 reductions on the GPU); with NULL it stays asynchronous. */
int pie_iteration(pie_ctx* ctx, void* object, int transform, double beta,
                  pie_stats* stats, void* stream);

/* pie_iteration in the given mode (PIE_MODE_COLOURED or PIE_MODE_BATCHED)
 * whatever the context was created with; the batched step divides by the
 * context's illumination as in batched contexts. A batched sweep on a
 * coloured context allocates one object-sized accumulator on first use. */
int pie_iteration_mode(pie_ctx* ctx, void* object, int transform, int mode, double beta,
                       pie_stats* stats, void* stream);

/* Blind PIE (Eq. pie_update with Eq. epie_probe_update), coloured mode only:
 * one sweep that also refines the context's probe. Within a colour every
 * position uses the probe of the colour's start and updates its patch; the
 * probe step of Eq. epie_probe_update is then evaluated at each updated patch,
 * g_j = conj(z_j) (w z_j - P_M(z_j)) (a second transform pair per position),
 * and after the colour w <- w - gamma sum_j g_j / (sum_j |z_j|^2 + delta),
 * delta = delta_rel max(sum_j |z_j|^2) (probe_step PIE_PROBE_STEP_NORMALISED)
 * or w <- w - gamma sum_j g_j (PIE_PROBE_STEP_SCALAR). The object step is
 * beta conj(w) / max|w|^2 with the probe of that colour. With one position per
 * colour (pie_ctx_set_order with one_per_colour) and the scalar step this is
 * Eq. pie_update and Eq. epie_probe_update exactly as stated, the probe
 * refined after every position in the visiting order. INVALID_ARG for
 * gamma < 0 or an unknown probe_step. */
int pie_iteration_blind(pie_ctx* ctx, void* object, int transform, double beta, double gamma, int probe_step,
                        pie_stats* stats, void* stream);

/* Copy the context's current probe into `probe_out` (device [n][n] complex),
 * or replace it with `probe` (device, copied; synchronises `stream`). */
int pie_ctx_probe(const pie_ctx* ctx, void* probe_out, void* stream);
int pie_ctx_set_probe(pie_ctx* ctx, const void* probe, void* stream);

/* Algorithm 3: PFT sweeps until rel_change < tol_pft or max_pft sweeps, then
 * full-FFT sweeps until rel_change < tol_full or max_full sweeps.
 * truth: optional device [obj_h][obj_w] complex; with it each trace entry also
 * holds the phase-aligned error on the illuminated mask (pixels with
 * illumination >= 1e-3 of its maximum). trace: host array with room for
 * max_pft + max_full entries (may be NULL); *ntrace receives the count.
 * Synchronises `stream` after every sweep (the stopping rule reads norms). */
typedef struct pie_schedule {
  double beta_pft, beta_full;
  double tol_pft, tol_full;
  int max_pft, max_full;
  double tv_pft, tv_full;  /* TV weights (0 = none): one pie_tv_step after each sweep */
  double tv_eps;           /* TV smoothing (0 = 1e-3)                                 */
  int pft_batched;         /* 1: PFT phase in PIE_MODE_BATCHED (one launch per sweep,
                              all positions read the same object), full phase in the
                              context's mode; 0: both phases in the context's mode   */
} pie_schedule;

typedef struct pie_trace {
  int phase;             /* PIE_TRANSFORM_PFT or PIE_TRANSFORM_FULL */
  double phi, rel_change, nrmse;
  double seconds;        /* wall time since the call started        */
} pie_trace;

int warm_start_then_refine(pie_ctx* ctx, void* object, const pie_schedule* schedule,
                           const void* truth, pie_trace* trace, int* ntrace, void* stream);

/* Total-variation regularisation (Section 4 regularises both phases with TV;
 * the term is not spelled out there). One gradient step on the smoothed
 * isotropic TV, in place on `object`:
 *   z <- z - lambda (D_x^H(D_x z / s) + D_y^H(D_y z / s)),
 *   s = sqrt(|D_x z|^2 + |D_y z|^2 + eps^2),
 * forward differences, zero flux across the last row and column. */
int pie_tv_step(pie_ctx* ctx, void* object, double lambda, double eps, void* stream);

/* Visiting order of the scan positions (the blind experiments of Section 4.2
 * draw a random order without replacement). order: host int32 [N], a
 * permutation of 0..N-1, or NULL for index order. With one_per_colour == 0
 * the positions are re-coloured greedily in that order and every sweep then
 * runs colour-major with that order inside each colour; with one_per_colour
 * != 0 every position is its own colour and sweeps visit the positions in
 * exactly that order (Section 2.1's sequential j; the dataflow launch form
 * still runs positions whose patches do not overlap at the same time).
 * Synchronises the device. */
int pie_ctx_set_order(pie_ctx* ctx, const int32_t* order, int one_per_colour);

/* Test hook for the error path of the bounded device waits. kind:
 * PIE_TEST_WAIT_GRID_BARRIER raises the target of every grid barrier of a
 * PIE_LAUNCH_PERSISTENT sweep by one, PIE_TEST_WAIT_DATAFLOW the completion
 * count every PIE_LAUNCH_DATAFLOW position waits for, so that wait can never
 * be met (no CTA ever adds the missing arrival); PIE_TEST_WAIT_NONE (normal
 * use) turns it off. The next sweep in that launch form then runs the wait's
 * 2 s timeout: the waiting CTA sets the sweep's error word, every other CTA
 * sees it and stops waiting, every cluster barrier is still matched, so the
 * launch ends with the object unspecified. A sweep called with `stats`
 * (which synchronises) returns PFT_ERR_TIMEOUT itself; otherwise the next
 * pie_iteration* or warm_start_then_refine call returns it. The call after
 * that runs normally. Synchronises the device when the setting changes. */
#define PIE_TEST_WAIT_NONE         0
#define PIE_TEST_WAIT_GRID_BARRIER 1
#define PIE_TEST_WAIT_DATAFLOW     2
int pie_ctx_test_unreachable_wait(pie_ctx* ctx, int kind);

/* How coloured sweeps of `transform` are launched (PIE_LAUNCH_*):
 * PIE_LAUNCH_PERSISTENT runs the whole sweep as one cooperative launch (the
 * fused kernel loops over the colours with a grid barrier in between; as many
 * clusters as fit on the GPU at once); PIE_LAUNCH_DATAFLOW is one cooperative
 * launch over the colour-major schedule in which each position waits, on
 * per-position completion counters, only for the earlier positions whose
 * patches overlap its own (transitively reduced at set-up), so positions of
 * consecutive colours run at the same time; PIE_LAUNCH_PER_COLOUR is one
 * launch per colour. Results are identical in all three (every patch is read
 * after all earlier overlapping positions wrote it and before any later one
 * does; the per-position arithmetic does not change). Waits are bounded
 * (2 s): a timeout is latched and returned by the next call as
 * PFT_ERR_TIMEOUT. The autotuner picks the fastest form (and, for the
 * dataflow form, its cluster size) at creation; INVALID_ARG for another
 * value, UNSUPPORTED in batched mode or when the transform is not built. If
 * the device refuses the cooperative launch, the next sweep falls back to one
 * launch per colour (pie_ctx_info_get shows it). */
int pie_ctx_set_persistent(pie_ctx* ctx, int transform, int persistent);

/* Cluster size (CTAs per position: 1, 2, 4 or 8) of `transform`'s sweeps in
 * the context's mode, in every launch form, in place of the autotuner's or
 * the built-in choice (largest size whose clusters for a whole colour fit on
 * the GPU at once); 0 returns to the built-in choice. The result of a sweep
 * does not depend on it beyond the rounding of the FP32 transforms (the
 * rows, columns and reductions are split differently over the CTAs).
 * INVALID_ARG for another value; UNSUPPORTED when no kernel of that size is
 * built for the context's (n, M) and mode. Synchronises the device. */
int pie_ctx_set_cluster(pie_ctx* ctx, int transform, int cluster);

/* Phase-aligned error min_phi ||e^{i phi} z - truth|| / ||truth|| over the
 * context's illuminated mask (FP64 on the GPU); synchronises `stream`. */
int pie_nrmse(pie_ctx* ctx, const void* object, const void* truth, double* out, void* stream);

/* Amplitude loss through the context's partial transform A:
 *   L = sum_j || |A(w . Q_j z)| - d_j^crop ||^2,
 * with gradients in the convention dL/dRe + i dL/dIm:
 *   grad_obj   device [obj_h][obj_w] complex (overwritten),
 *   grad_probe device [n][n] complex (overwritten, may be NULL),
 * for the given object and probe (device, not modified). The exit waves are
 * recomputed per position, not stored. *loss (host) is written after a
 * synchronisation of `stream`. */
int pie_amp_loss_grad(pie_ctx* ctx, const void* object, const void* probe, void* grad_obj,
                      void* grad_probe, double* loss, void* stream);

/* ---- many independent reconstructions ------------------------------------
 * A batch holds `count` independent PIE problems whose sizes may differ (the
 * object, probe, scan and output size of each instance are its own). One call
 * sweeps every position of every instance: instances with the same (n, M) form
 * a shape class whose positions share one kernel launch per colour (coloured
 * mode in the default PIE_LAUNCH_PER_COLOUR form: launch c runs colour c of all
 * of them) or one launch per sweep (batched mode, and coloured mode in the
 * PIE_LAUNCH_DATAFLOW form: the class's colour-major work list in one launch,
 * each position waiting only for the earlier positions of its own instance
 * whose patches overlap its own, with clusters claiming positions in list
 * order so that the classes' launches can share the GPU in any proportion).
 * The two coloured forms give the same objects. The classes run as parallel
 * branches of one CUDA graph, captured on first use and replayed.
 *
 * pie_batch_create(out, count, problems, probes, positions, intensities, stream)
 *   problems: host [count] (all with the same mode; `autotune` is ignored);
 *   probes, positions, intensities: host arrays of `count` pointers, each as
 *   for pie_ctx_create. Synchronises `stream`.
 * pie_batch_iteration(b, objects, transform, beta, phi, stream)
 *   objects: host array of `count` device object pointers (updated in place);
 *   phi: host double [count] or NULL; with it the call synchronises and
 *   writes each instance's Phi (as pie_stats.phi).
 * pie_batch_classes: number of shape classes and kernel launches per sweep.
 * pie_batch_set_launch(b, form): PIE_LAUNCH_PER_COLOUR (default) or
 *   PIE_LAUNCH_DATAFLOW for a coloured batch (INVALID_ARG for another form,
 *   UNSUPPORTED for a batched-mode batch); synchronises the device. A wait that
 *   gives up (2 s) is returned as PFT_ERR_TIMEOUT by the call that sees it.
 */
typedef struct pie_batch pie_batch;

int pie_batch_create(pie_batch** out, int count, const pie_problem* problems, const void* const* probes,
                     const int32_t* const* positions, const float* const* intensities, void* stream);
int pie_batch_destroy(pie_batch* batch);
int pie_batch_iteration(pie_batch* batch, void* const* objects, int transform, double beta, double* phi,
                        void* stream);
int pie_batch_classes(const pie_batch* batch, int* nclasses, int* launches_per_sweep);
int pie_batch_set_launch(pie_batch* batch, int form);

/* ---- PIE over large frames ----------------------------------------------
 * Section 4's large-scale regime (frames of n = 2048 ... 16384 pixels a side,
 * M = 128): the PFT sweeps of Algorithm 3's warm-start phase (Eq. pie_update
 * with the PFT of Algorithm 5 and reading R4 for its inverse), coloured, on
 * the split-BF16 large-frame transforms. Each colour's positions (disjoint
 * patches) are one batch: exit waves w . Q_j z, pft_forward, the modulus
 * projection onto the cropped amplitudes, pft_adjoint, and the object update
 * beta conj(w) / (max|w|^2 n^2) A^H R. A sweep is sequential PIE in
 * colour-major order (greedy colouring in index order, as pie_scan_schedule).
 * The full-FFT refine phase is not built for these sizes.
 *
 * pie_lf_create(out, problem, probe, positions, intensities, stream)
 *   problem: as for pie_ctx_create; mode must be PIE_MODE_COLOURED, the
 *   object width even, n and M a large-frame shape pft_plan_create builds in
 *   PFT_PREC_SPLIT_BF16 (n = 2048 ... 16384, M = 128), else UNSUPPORTED.
 *   probe: device [n][n] complex (copied); positions: host int32 [N][2]
 *   (row, col), patches inside the object, every col even (INVALID_ARG
 *   otherwise); intensities: device float [N][n][n] in FFT order, of which
 *   only the centred M x M crop is kept (sqrt taken); a NaN or infinite value
 *   returns PFT_ERR_NONFINITE. Synchronises `stream`.
 * pie_lf_iteration(ctx, object, beta, stats, stream)
 *   one PFT sweep in place on `object` (device [obj_h][obj_w] complex,
 *   16-byte aligned). With `stats` the call synchronises and fills Phi (Eq. 4
 *   by R12) and the relative change (allocating one object-sized copy on
 *   first use); NONFINITE for a non-finite objective or change.
 * pie_lf_colours(ctx, ncolours, max_colour): colours and the largest colour.
 */
typedef struct pie_lf pie_lf;

int pie_lf_create(pie_lf** out, const pie_problem* problem, const void* probe, const int32_t* positions,
                  const float* intensities, void* stream);
int pie_lf_destroy(pie_lf* ctx);
int pie_lf_iteration(pie_lf* ctx, void* object, double beta, pie_stats* stats, void* stream);
int pie_lf_colours(const pie_lf* ctx, int* ncolours, int* max_colour);

/* ---- allocation-free error reduction ------------------------------------
 * The paper has no counterpart to this call. It exists for callers that cannot
 * call cudaMalloc when they need the error: plug-ins inside a host framework
 * that owns every device allocation through its own pool (an allocation made
 * behind the pool's back breaks its accounting or is refused), and
 * latency-critical loops, where cudaMalloc / cudaFree can synchronise the
 * whole device.
 *
 * pie_nrmse_noalloc(object, truth, mask, count, out, stream)
 *   Same quantity as pie_nrmse, min_phi ||e^{i phi} z - truth|| / ||truth||,
 *   over the elements whose mask byte is non-zero (mask == NULL: all).
 *   object, truth: device complex [count]; mask: device uint8 [count] or NULL;
 *   out: host double. 1 <= count <= 16,777,216 (a 4096 x 4096 object); larger
 *   counts return PFT_ERR_INVALID_ARG before any GPU work. Two passes on the
 *   device (the aligning phase, then the sum of |e^{i phi} z - truth|^2), then
 *   the call copies the result to the host and synchronises `stream`.
 *   It calls no allocator (no cudaMalloc, no cudaFree, no library routine that
 *   allocates): its partial sums live in a fixed 128 KiB array compiled into
 *   the library, held on every GPU that loads the library until the process
 *   exits.
 *   Set-up: the first call on a device, with that device current, looks up the
 *   array's device address (cudaGetSymbolAddress, which can load the library's
 *   device code on that device) and keeps it; make that first call before any
 *   stream capture begins, since the lookup is a CUDA call that a capture in
 *   progress may refuse (the call then returns PFT_ERR_CUDA). The kept address
 *   is not refreshed after cudaDeviceReset; do not use the call on a device
 *   after resetting it.
 *   All calls share the array and each call leaves its sums in it; every slot a
 *   call reads is written earlier by the same call. Calls that overlap on the
 *   GPU (other streams, other host threads) race on the array and must be
 *   serialised by the caller.
 */
int pie_nrmse_noalloc(const void* object, const void* truth, const uint8_t* mask, int64_t count,
                      double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PFT_GB300_H */
