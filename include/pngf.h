/*
 * pngf.h - C ABI of the PNGF direct-binary-search (DBS) hot path on one GPU.
 *
 * Method (arXiv 2501.18054, "Near real-time full-wave inverse design of
 * electromagnetic devices"): a precomputed numerical Green function G (Eq. 3)
 * reduces the evaluation of a candidate design to a linear system over the
 * design region only (Eqs. 2 and 7; generalised materials and the field form
 * in Supplementary Note 4).  DBS flips one pixel at a time and keeps the flip
 * if the objective improves (section "Direct binary search optimization",
 * Supplementary Fig. 1).  A flip is a rank-1 change of the system matrix, so
 * every candidate is scored exactly through the Woodbury / Sherman-Morrison
 * identity (Eq. 9, scored through R and S as in Eqs. 11-14) and the maintained
 * inverse is corrected rank-1 when a flip is kept (Eq. 9; cost in
 * Supplementary Note 3).
 *
 * Field-form notation used throughout (one unknown per pixel, 2D TM):
 *   G    = G_dd   (n_d x n_d)  design-to-design Green function, complex symmetric
 *   G_od          (n_o x n_d)  design-to-port functionals (the paper's G_obj)
 *   c_d, c_o                   incident field on the pixels / at the ports
 *                              (the paper's e_inc and x_inc)
 *   v_k  = dv_k * b_k          contrast of pixel k, b in {0,1}^n_d (the
 *                              paper's Y, Supplementary Note 4)
 *   M    = I - G diag(v)       reduced system, M e = c_d
 *   o    = c_o + G_od (v .* e) port amplitudes (the paper's x_obj, Eq. 5)
 *   S_p  = (o_p - s_off_p) * s_scale_p,  f = objective(S)
 *   W    = M^-1 G              maintained inverse (the paper's C~^-1 of the
 *                              field form, Supplementary Note 4)
 *   T    = G_od (I + V W)      port projection of W (the paper's R, Eq. 11)
 * Flipping pixel k changes v_k by delta; with d_k = 1 - delta W_kk and
 * alpha = delta / d_k the candidate ports are o + alpha e_k T[:,k] (Eq. 14)
 * and an accepted flip applies W += alpha c c^T, c = W[:,k] (Eq. 9).
 *
 * Conventions of every call:
 *  - Complex numbers are interleaved (re, im) doubles: "c128".
 *  - Every array pointer is a DEVICE pointer unless its comment says "host".
 *    The caller owns every array.  The library keeps the pointers to G_dd,
 *    G_od, c_d, c_o and dv given to pngf_create; they must stay valid and
 *    unchanged until pngf_destroy.  It allocates no device memory: all scratch
 *    lives in the caller's workspace (size from pngf_workspace_size).
 *  - Work is ordered on the stream given to pngf_create.  Calls returning
 *    device results do not synchronize; calls with host outputs do.
 *  - Every call returns a pngf_status and never aborts the process.  A
 *    failure detected on the device (singular pivot, non-finite value, a wait
 *    that timed out) is latched in the workspace and returned by the next call
 *    that synchronizes (pngf_eval_ports, pngf_sync).
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef PNGF_H
#define PNGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* pngf_stream; /* a cudaStream_t; NULL = default stream */
typedef struct pngf_ctx pngf_ctx;        /* opaque, host-side handle */

typedef enum {
  PNGF_OK = 0,
  PNGF_EINVAL = 1,        /* bad argument (size, pointer, alignment, mode) */
  PNGF_ENOMEM = 2,        /* workspace smaller than pngf_workspace_size */
  PNGF_ECUDA = 3,         /* a CUDA runtime call failed */
  PNGF_ESINGULAR = 4,     /* zero pivot in the factorisation of M */
  PNGF_ENOTFACTORED = 5,  /* pngf_factor has not run on this context */
  PNGF_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
  PNGF_ENUMERIC = 7,      /* non-finite value met on the device */
  PNGF_ECAPACITY = 8,     /* trace buffer full (kept flips past it are applied, not recorded) */
  PNGF_EACCURACY = 9      /* PNGF_MIXED: a refresh found the field's residual above 1e-3 of the
                             field (the FP32 maintained inverse lost accuracy: an ill-conditioned
                             system, such as a design driven into a high-Q resonance); the search
                             stops and its state is not to be trusted: use PNGF_FP64 */
} pngf_status;

/* PNGF_FP64: every step in FP64.  PNGF_MIXED: an FP32 maintained inverse with a
 * delayed rank-delay_r correction, the decision state (diag W, e, T, o, f) as
 * FP32 pairs (~48 bits, FP32 exponent range: magnitudes and their squares must
 * stay within about 1e+-38), refreshed against G every refresh_k flips.
 * PNGF_PEC: FP64, pixels of perfect electric conductor (the paper's binary
 * system, Eq. 2, [(I - P) + P G] j = P e_inc; dv is not used): the search
 * keeps H = (G_MM)^-1 of the metal set M, Q = G H and W = G - G H G, and a
 * flip is a symmetric rank-1 change of H and W and a rank-1 change of Q; the
 * state of a design is built from the empty design by rank-1 additions
 * (pngf_factor).  No refresh (refresh_k is ignored); pngf_set_state,
 * pngf_gradient, pngf_score_flips' o_new, the batch and tile calls are not
 * available (PNGF_EINVAL).  pngf_get_state returns W (upper triangle current),
 * diag W, the total field e (zero on metal) and T = G_od - G_od H G. */
typedef enum { PNGF_FP64 = 0, PNGF_MIXED = 1, PNGF_PEC = 2 } pngf_precision;
typedef enum { PNGF_FIRST_IMPROVEMENT = 0, PNGF_BEST_IMPROVEMENT = 1 } pngf_dbs_mode;
typedef enum {
  PNGF_OBJ_MAX_WEIGHTED_POWER = 0, /* maximise sum_p w_p |S_p|^2 */
  PNGF_OBJ_MIN_INSERTION_LOSS = 1  /* minimise sum_p w_p (1 - |S_p|)^2 (Supplementary Note 9) */
} pngf_objective;

#define PNGF_MAX_PORTS 8

typedef struct {
  int32_t n_d;        /* design pixels, 1 <= n_d <= 32768 */
  int32_t n_o;        /* ports, 1 <= n_o <= PNGF_MAX_PORTS */
  int32_t precision;  /* pngf_precision */
  int32_t mode;       /* pngf_dbs_mode */
  int32_t objective;  /* pngf_objective */
  int32_t refresh_k;  /* iterative-refinement refresh of e, T, o every refresh_k accepted
                         flips (0 = never): residual against G in FP64 (PNGF_FP64) or in
                         FP32-pair arithmetic (PNGF_MIXED, a multiple of delay_r) */
  int32_t delay_r;    /* PNGF_MIXED: flips accumulated before the maintained inverse is
                         updated in one rank-delay_r product (1..128); ignored for FP64 */
  int32_t n_ctas;     /* persistent sweep grid (0 = one per SM, capped by occupancy) */
  double tau;         /* accept iff gain > tau * max(|f|, 1e-30) */
  double obj_weights[PNGF_MAX_PORTS]; /* w_p */
  double s_off[2 * PNGF_MAX_PORTS];   /* c128 per port */
  double s_scale[2 * PNGF_MAX_PORTS]; /* c128 per port, nonzero for p < n_o */
  int32_t tensor_fold; /* PNGF_MIXED: 1 = fold the delayed set into the FP32 inverse on the
                          tensor cores (tcgen05, 3xTF32), 0 = FP32 CUDA cores */
  int32_t reserved;
} pngf_config;

/* Bytes of device workspace a context with this configuration needs. */
pngf_status pngf_workspace_size(const pngf_config* cfg, size_t* bytes);

/*
 * Bind the precomputed inputs (Eqs. 3 and 5; section "Precomputation"):
 *   G_dd  c128 n_d x n_d row-major, complex symmetric (reciprocal background)
 *   G_od  c128 n_o x n_d row-major
 *   c_d   c128 n_d;  c_o  c128 n_o
 *   dv    c128 n_d: contrast of a pixel that is "on" (k^2 (eps_on - eps_off))
 * workspace: >= pngf_workspace_size bytes, 256-byte aligned, device memory.
 * Nothing is computed until pngf_factor.  *out receives a host handle.
 */
pngf_status pngf_create(const pngf_config* cfg, const double* G_dd, const double* G_od,
                        const double* c_d, const double* c_o, const double* dv,
                        void* workspace, size_t workspace_bytes, pngf_stream stream,
                        pngf_ctx** out);

/*
 * Factor M = I - G diag(dv .* b) once (blocked LU with partial pivoting, FP64)
 * and form the maintained state W = M^-1 G, e = M^-1 c_d, T = G_od (I + V W),
 * o = c_o + G_od (v .* e) (the paper's initial inversion of C_0,
 * section "Direct binary search optimization").  b: uint8 n_d (0/1).
 * Returns PNGF_ESINGULAR (via the latched status) if a pivot is exactly 0.
 */
pngf_status pngf_factor(pngf_ctx* ctx, const uint8_t* b);

/*
 * Score candidate flips against the current state without changing it
 * (Eq. 14): for each listed pixel k, f_new[i] = objective after flipping k.
 *   pixels  int32 n (device), 0 <= pixels[i] < n_d
 *   f_new   double n (device, out)
 *   o_new   c128 n x n_o (device, out) or NULL
 * A candidate with |d_k| < 1e-14 gets f_new = NaN.
 */
pngf_status pngf_score_flips(pngf_ctx* ctx, const int32_t* pixels, int32_t n, double* f_new,
                             double* o_new);

/* Keep the flip of one pixel: rank-1 update of W, T, e, o, v, b (Eq. 9). */
pngf_status pngf_accept_flip(pngf_ctx* ctx, int32_t pixel);

/*
 * pngf_accept_flip for callers that cannot allocate device memory: the same
 * kept-flip update, but its scratch (the pivot record and the gathered
 * column of W) lives in a fixed array inside the library instead of the
 * workspace.  It exists for callers that may not allocate device memory
 * while they run: code whose device memory was reserved up front by another
 * component (a framework's caching allocator that owns the whole pool), or a
 * latency-bound loop that must not block on the device-wide synchronisation a
 * cudaMalloc or cudaFree can imply.  Such callers set up the context and its
 * workspace once, beforehand, and then only pass it in.  The paper has no
 * counterpart to this entry point.
 *
 *   - FP64 contexts only, and n_d <= PNGF_NOALLOC_MAX_ND (8192), else
 *     PNGF_EINVAL; the context's device must be the current device.
 *   - The array (256 + 16 * PNGF_NOALLOC_MAX_ND bytes, about 128 KiB) is held
 *     by every GPU that loads the library, until the process exits.
 *   - The first call on a device looks the array's device address up once
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call and every context share the one array: calls that overlap on
 *     the GPU (other streams, other contexts) race with each other; order them
 *     on one stream.  Each call overwrites the array before it reads it.
 *   - It allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 */
#define PNGF_NOALLOC_MAX_ND 8192
pngf_status pngf_accept_flip_noalloc(pngf_ctx* ctx, int32_t pixel);

/*
 * Run direct binary search on the device (section "Direct binary search
 * optimization" and Supplementary Fig. 1: flip a tile, evaluate, keep the flip
 * if the objective improved, else try another; converged when every flip was
 * tried without improvement), each candidate scored by Eq. 14 and each kept
 * flip applied by Eq. 9: up to n_sweeps passes over the pixels; a pass that
 * keeps no flip ends the search (converged).
 *   order     int32 n_sweeps x n_d (device): visiting order of each pass, each
 *             row a permutation of 0..n_d-1; NULL = raster order 0..n_d-1.
 *             FIRST mode keeps the first improving flip in visiting order
 *             (sequential DBS semantics); BEST mode keeps the best improving
 *             flip of the whole region per step (ties -> lowest pixel index),
 *             ignores order, and n_sweeps bounds its number of steps (each
 *             step evaluates all n_d pixels).
 *   trace     int32 trace_cap x 4 (device, out): per kept flip
 *             (sweep, position, pixel, 0); may be NULL if trace_cap == 0
 *   trace_f   double trace_cap (device, out): objective after each kept flip, or NULL
 *   counters  int64 8 (device, out): [0] kept flips, [1] attempted flips
 *             (evaluations in sequential semantics), [2] sweeps run,
 *             [3] converged (0/1), [4] refreshes, [5] flushes, [6] status,
 *             [7] active pixels (b_i = 1) summed over the refreshes
 * Kept flips past trace_cap are still applied but not recorded; [6] is then
 * PNGF_ECAPACITY.  The state stays on the device for further calls.
 * Mixed precision keeps each CTA's share of the pixels in shared memory:
 * with own = ceil(N_d / grid) (grid = one CTA per SM, or n_ctas) rounded up
 * to 32, own <= 256 and (delay_r + 8) x own x 8 bytes <= 144 KiB (the
 * delayed rows and partial sums), else PNGF_EINVAL before any launch.
 */
pngf_status pngf_dbs_sweep(pngf_ctx* ctx, int32_t n_sweeps, const int32_t* order,
                           int32_t* trace, double* trace_f, int32_t trace_cap,
                           int64_t* counters);

/*
 * Batched DBS: many independent runs advanced by one kernel launch, one CTA
 * per run at a time.  Independent systems exchange nothing: section
 * "Computational efficiency" (and Table 1's footnote on multi-frequency
 * designs) notes that the systems of different frequencies are independent and
 * can be advanced in parallel; here they are independent random starts and/or
 * design regions of different sizes sharing one device.  Each run is the
 * search of pngf_dbs_sweep (section "Direct binary search optimization").
 *   ctxs      host array of n_ctx factored contexts (1 <= n_ctx <= PNGF_BATCH_MAX_RUNS),
 *             one device, one precision and mode, n_d <= PNGF_BATCH_MAX_ND each;
 *             the launch goes to ctxs[0]'s stream, which must order every
 *             context's earlier work
 *   orders    host array of n_ctx device pointers (each as pngf_dbs_sweep's
 *             order, NULL = raster), or NULL for raster everywhere
 *   traces, trace_f   host arrays of n_ctx device pointers, or NULL
 *   trace_cap capacity of every trace
 *   counters  int64 n_ctx x 8 (device, out), per run as in pngf_dbs_sweep
 *   batch_ws  device scratch of pngf_batch_workspace_size(n_ctx) bytes, 256-byte aligned
 * Each run follows the same semantics as pngf_dbs_sweep on its own context.
 * Scheduling (no effect on the results): one CTA per SM takes the runs from a
 * queue in descending n_d (ties in the given order), so that the largest runs
 * start first, each on an SM of its own.
 */
/* n_d <= PNGF_BATCH_MAX_ND for every run: the FP64 batch kernel stages one
 * run's gathered column and the column times alpha in 32 x n_d bytes of shared
 * memory (128 KiB at the bound), so a larger region returns PNGF_EINVAL before
 * any launch. */
#define PNGF_BATCH_MAX_RUNS 65536
#define PNGF_BATCH_MAX_ND 4096
pngf_status pngf_batch_workspace_size(int32_t n_ctx, size_t* bytes);
pngf_status pngf_dbs_sweep_batch(pngf_ctx* const* ctxs, int32_t n_ctx, int32_t n_sweeps,
                                 const int32_t* const* orders, int32_t* const* traces,
                                 double* const* trace_f, int32_t trace_cap, int64_t* counters,
                                 void* batch_ws, size_t batch_ws_bytes);

/*
 * Tile flips on one or several systems (FP64).
 *
 * A candidate flips every pixel of one tile at once: the paper's tile flips of
 * M unknowns (section "Low-rank update evaluation": dP_n = Q^T H_P Q, scored
 * by Eq. 14 and kept by the rank-M Woodbury update of Eq. 9; its designs flip
 * 2 to 4 symmetry-tied tiles together, Methods, "Optimization parameters").
 * In field form, for tile K of m pixels with contrast changes D:
 *   A = I - D W_KK (m x m), score o + T[:, K] A^-1 D e_K,
 *   keep W += U Z U^T with U = W[:, K], Z = A^-1 D (and e, T, diag W, b, v).
 * Several systems -- one per frequency: the paper precomputes G, G_obj and
 * C^-1 per frequency and updates them independently ("Computational
 * efficiency") -- share the design; every candidate is scored in every system
 * and the objectives are combined into one (Supplementary Note 9: a mean or a
 * min-max rule), which decides with the first system's tau.
 *
 *   ctxs     host array of n_sys contexts (1..PNGF_TILES_MAX_SYSTEMS), all FP64,
 *            factored at the same design, same n_d, objective kind and mode and
 *            device; the launch goes to ctxs[0]'s stream, which must order
 *            every context's earlier work; refresh_k and n_ctas of ctxs[0] apply;
 *            device-side errors are latched in ctxs[0]
 *   combine  pngf_combine
 *   tiles    int32 n_tiles x tile_m (device): the distinct pixels of each tile,
 *            -1 entries pad (1 <= tile_m <= PNGF_TILE_MAX); an entry outside
 *            [-1, n_d) latches PNGF_EINVAL
 *   ws       device scratch of pngf_tiles_workspace_size bytes, 256-byte aligned
 * A candidate whose m x m system meets a pivot below 1e-14 in magnitude (in
 * any system) is skipped, as |d_k| < 1e-14 is for single pixels.
 */
#define PNGF_TILES_MAX_SYSTEMS 4
#define PNGF_TILE_MAX 16
typedef enum {
  PNGF_COMBINE_MEAN = 0, /* arithmetic mean of the systems' objectives */
  PNGF_COMBINE_WORST = 1 /* the worst system: min of maximised, max of minimised objectives */
} pngf_combine;

pngf_status pngf_tiles_workspace_size(int32_t n_sys, int32_t n_d, int32_t n_tiles, int32_t tile_m,
                                      size_t* bytes);

/* DBS over tiles with pngf_dbs_sweep's semantics, tiles in place of pixels:
 * order int32 n_sweeps x n_tiles (device, rows permutations of the tile
 * indices) or NULL (0..n_tiles-1); trace entries (sweep, position, tile, 0),
 * trace_f the combined objective after each kept flip; counters as
 * pngf_dbs_sweep's ([5] = 0).  Each context's own port amplitudes and
 * objective are updated (pngf_eval_ports). */
pngf_status pngf_dbs_sweep_tiles(pngf_ctx* const* ctxs, int32_t n_sys, int32_t combine, const int32_t* tiles,
                                 int32_t n_tiles, int32_t tile_m, int32_t n_sweeps, const int32_t* order,
                                 int32_t* trace, double* trace_f, int32_t trace_cap, int64_t* counters,
                                 void* ws, size_t ws_bytes);

/* Score listed tiles without changing the state: list int32 count (device,
 * tile indices), F double count (device, out: combined objective, NaN if
 * singular), f_sys double count x n_sys (device, out, or NULL). */
pngf_status pngf_score_tiles(pngf_ctx* const* ctxs, int32_t n_sys, int32_t combine, const int32_t* tiles,
                             int32_t n_tiles, int32_t tile_m, const int32_t* list, int32_t count, double* F,
                             double* f_sys, void* ws, size_t ws_bytes);

/* Keep the flip of one tile in every system (the rank-m update); a singular
 * tile latches PNGF_ESINGULAR in ctxs[0] and changes nothing. */
pngf_status pngf_accept_tile(pngf_ctx* const* ctxs, int32_t n_sys, int32_t combine, const int32_t* tiles,
                             int32_t n_tiles, int32_t tile_m, int32_t tile, void* ws, size_t ws_bytes);

/* Current port amplitudes x_obj (c128 n_o, host; Eq. 5, o = c_o + G_od (v .* e))
 * and objective of the S-parameters (host; the objective forms of
 * Supplementary Note 9); synchronizes. */
pngf_status pngf_eval_ports(pngf_ctx* ctx, double* o_host, double* f_host);

/* Copy the current design (uint8 n_d, device). */
pngf_status pngf_get_design(pngf_ctx* ctx, uint8_t* b);

/*
 * Read back the maintained state: the quantities the paper keeps between
 * iterations (C^-1, R and S of Eqs. 11-13, in field form W, T and e) and the
 * current x_obj (device outputs, any may be NULL):
 *   W c128 n_d x n_d (FP64 precision only, else PNGF_EINVAL if non-NULL; only
 *     the upper triangle j >= i is current, the rest is as the search left it),
 *   diag_W c128 n_d, e c128 n_d, T c128 n_o x n_d, o c128 n_o.
 */
pngf_status pngf_get_state(pngf_ctx* ctx, double* W, double* diag_W, double* e, double* T,
                           double* o);

/*
 * Gradient of the objective with respect to a continuous density rho_m of
 * every pixel (v_m = rho_m dv_m; rho = b is the current binary design), from
 * the maintained state alone (Supplementary Note 5, the chain rule with
 * Wirtinger derivatives in its elementwise O(N_obj) form, here in the field
 * form where dx_obj/dv_m = T[:, m] e_m):
 *   grad    double n_d (device, out): df/drho_m = 2 Re[sum_p (dphi_p/dS_p) scale_p T[p,m] e_m dv_m]
 *   dodrho  c128 n_o x n_d (device, out) or NULL: do_p/drho_m = T[p,m] e_m dv_m
 * dphi/dS = w conj(S) (PNGF_OBJ_MAX_WEIGHTED_POWER) or -w (1 - |S|) conj(S)/|S|
 * (PNGF_OBJ_MIN_INSERTION_LOSS; 0 where S = 0).  Either precision (the mixed
 * path's e and T are its FP64 copies, current after every call).
 */
pngf_status pngf_gradient(pngf_ctx* ctx, double* grad, double* dodrho);

/* Kept flips since the last refresh (host int32); synchronizes.  Part of a
 * checkpoint: with it, a resumed search refreshes where the original would. */
pngf_status pngf_get_since_refresh(pngf_ctx* ctx, int32_t* since_refresh);

/*
 * Checkpoint import: replace the maintained state of a factored context by one
 * that pngf_get_state / pngf_get_design / pngf_get_since_refresh exported,
 * possibly from another process (the paper's maintained C^-1, R, S, x_obj of
 * Eqs. 11-13 between two iterations; the checkpoint itself has no counterpart
 * in the paper).  Device inputs in the layouts pngf_get_state writes:
 *   b uint8 n_d, W c128 n_d x n_d (upper triangle read), diag_W, e c128 n_d,
 *   T c128 n_o x n_d, o c128 n_o; since_refresh >= 0.
 * FP64 contexts: b and W are required; the context must have been created
 * with the same inputs and configuration and factored once (at any design);
 * the resumed search is then bit-for-bit the uninterrupted one.
 * Mixed contexts: b and W must be NULL and since_refresh < refresh_k; the
 * context must have been factored at the checkpoint's design; diag W, e, T
 * and o are replaced, the FP32 inverse is the factor's.
 * The objective is recomputed from o on the device; v follows b.
 */
pngf_status pngf_set_state(pngf_ctx* ctx, const uint8_t* b, const double* W, const double* diag_W,
                           const double* e, const double* T, const double* o,
                           int32_t since_refresh);

/*
 * Failure-detection controls (the paper has no counterpart).
 *   wait_log2  every bounded device-side wait of this context's later
 *              launches on other CTAs (grid barriers, the word polls of the
 *              mixed search) gives up after 2^wait_log2 polls and latches
 *              PNGF_ETIMEOUT (8..30; 0 = the default 2^24, about ten seconds)
 *   hold_cta   >= 0: CTA hold_cta of the next pngf_dbs_sweep waits, before it
 *              takes part in anything grid-wide, on a flag that nothing sets
 *              (bounded by the same limit); the other CTAs' waits for it run
 *              out, the call ends with PNGF_ETIMEOUT latched, nothing faults.
 *              One-shot.  -1 = none.
 * After a timeout the search state is undefined (restore a snapshot or factor
 * again); pngf_sync returns and clears the latched status.  Ordered on the
 * context's stream.
 */
pngf_status pngf_set_wait_limit(pngf_ctx* ctx, int32_t wait_log2, int32_t hold_cta);

/* Save the current state inside the workspace / restore it (same stream). */
pngf_status pngf_snapshot(pngf_ctx* ctx);
pngf_status pngf_restore(pngf_ctx* ctx);

/*
 * Tracing: SM clock cycles that CTA 0 of the last pngf_dbs_sweep spent per
 * phase, host int64 x 16: [0] scoring, [1] wait after scoring, [2] selection,
 * pivot and column gather, [3] wait before the update (FP64) / flush of the
 * delayed set (mixed), [4] state update (and the rank-1 update of W on the
 * FP64 path), [5] refreshes, [6] sweep set-up, [7] whole kernel,
 * [8..11] refresh sub-phases (x, residual, correction, ports), [12..15] 0.
 * Synchronizes the stream.
 */
pngf_status pngf_get_phase_cycles(pngf_ctx* ctx, int64_t* host16);

/*
 * Launch settings of later searches on this context (no counterpart in the
 * paper; what an autotuner varies between timed trials without re-factoring):
 *   n_ctas       persistent grid of pngf_dbs_sweep (0 = one per SM, as at create)
 *   tensor_fold  PNGF_MIXED: 1 = fold the delayed set on the tensor cores,
 *                0 = on the FP32 CUDA cores; must be 0 for FP64 contexts
 * The search state is untouched; call between searches, on the context's stream.
 */
pngf_status pngf_set_launch(pngf_ctx* ctx, int32_t n_ctas, int32_t tensor_fold);

/* Synchronize the stream and return the latched device status (then clear it). */
pngf_status pngf_sync(pngf_ctx* ctx);

const char* pngf_status_string(pngf_status s);
void pngf_destroy(pngf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PNGF_H */
