// C ABI entry points (include/pngf.h): argument checks, workspace layout and
// dispatch to the kernels of factor.cu and sweep.cu.  No entry point
// allocates device memory; all scratch is carved from the caller's workspace.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "flush_tc.cuh"

namespace pngf {

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

Layout make_layout(const pngf_config& cfg) {
  Layout L{};
  const size_t n = (size_t)cfg.n_d, n_o = (size_t)cfg.n_o;
  const bool mixed = cfg.precision == PNGF_MIXED;
  const bool pec = cfg.precision == PNGF_PEC;
  L.ldw = (int)align_up(n + 1, 8);
  L.ldl = (int)align_up(n, 32);
  L.ldt = (int)align_up(n, 8);
  L.R = mixed ? cfg.delay_r : 0;
  L.n_part = 1024;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t c = sizeof(c128);
  L.W = take(n * L.ldw * c);
  L.LU = take(n * L.ldw * c);  // PEC: H = (G_MM)^-1 padded
  L.Q = take(pec ? n * L.ldw * c : 0);  // PEC: Q = G H (full)
  // mixed path: [Wlo_re | Wlo_im | X | xa] contiguous, so one copy snapshots them
  const size_t plane = n * L.ldl * sizeof(float);
  L.Wlo_re = take(mixed ? 2 * plane : 0);
  L.Wlo_im = L.Wlo_re + (mixed ? plane : 0);
  L.X = take(n * (size_t)L.R * 2 * sizeof(float));
  L.xa = take((size_t)L.R * c);
  L.snapW_bytes = mixed ? off - L.Wlo_re : pec ? off - L.W : n * L.ldw * c;  // PEC: W, H, Q contiguous
  // contiguous state block: diag, e, T, v, b
  L.diag = off;
  off += align_up(n * c, 256);
  L.e = off;
  off += align_up(n * c, 256);
  L.T = off;
  off += align_up(n_o * L.ldt * c, 256);
  L.v = off;
  off += align_up(n * c, 256);
  L.b = off;
  off += align_up(n, 256);
  if (pec) {  // PEC: current j, R = G_od H, diag H
    L.pj = off;
    off += align_up(n * c, 256);
    L.pR = off;
    off += align_up(n_o * L.ldt * c, 256);
    L.pdiagH = off;
    off += align_up(n * c, 256);
  }
  L.state_bytes = off - L.diag;
  L.pos_of = take(n * sizeof(int));
  L.part = take((size_t)L.n_part * (2 * sizeof(long long) + 2 * sizeof(double) + kMaxPorts * c));
  L.rec = take((size_t)2 * L.n_part * kRecordBytes);
  L.slots = take((size_t)2 * L.n_part * 128);  // [2][P] one 128-B line per CTA
  if (mixed) {
    const size_t nk = (size_t)(L.R + TC_KC - 1) / TC_KC;
    L.tcimgA_bytes = (size_t)((n + TC_M - 1) / TC_M) * nk * TC_ACHUNK;
    L.tcimg_bytes = tc_image_bytes((int)n, L.R);
  }
  L.tcimg = take(L.tcimg_bytes);
  L.cbuf = take(n * c);
  L.rbuf = take(4 * (1 + n_o) * n * c + 1024);
  L.actg = take(n * sizeof(int));  // active-pixel list of the refresh
  L.gsum = take(pec ? 0 : n * n * sizeof(double));  // Re G + Im G (three-multiplication refresh products)
  // mixed path: G as FP32 pairs (double-float refresh residual) and the split refined vectors
  L.gsplit = take(mixed ? n * n * 4 * sizeof(float) : 0);
  L.xs = take(mixed ? (1 + n_o) * n * 8 * sizeof(float) : 0);
  L.xadd = take(mixed ? (size_t)L.R * 4 * sizeof(float) : 0);  // alpha_i of the mixed search as double-words
  L.ipiv = take(2 * n * sizeof(int));
  L.snapW = take(L.snapW_bytes);
  L.snapState = take(L.state_bytes + sizeof(Control));
  L.ctl = take(sizeof(Control));
  L.total = off;
  return L;
}

static pngf_status check_config(const pngf_config* cfg) {
  if (!cfg) return PNGF_EINVAL;
  if (cfg->n_d < 1 || cfg->n_d > 32768) return PNGF_EINVAL;
  if (cfg->n_o < 1 || cfg->n_o > PNGF_MAX_PORTS) return PNGF_EINVAL;
  if (cfg->precision != PNGF_FP64 && cfg->precision != PNGF_MIXED && cfg->precision != PNGF_PEC) return PNGF_EINVAL;
  if (cfg->mode != PNGF_FIRST_IMPROVEMENT && cfg->mode != PNGF_BEST_IMPROVEMENT) return PNGF_EINVAL;
  if (cfg->objective != PNGF_OBJ_MAX_WEIGHTED_POWER && cfg->objective != PNGF_OBJ_MIN_INSERTION_LOSS)
    return PNGF_EINVAL;
  if (cfg->refresh_k < 0) return PNGF_EINVAL;
  if (cfg->precision == PNGF_MIXED) {
    if (cfg->delay_r < 1 || cfg->delay_r > 128) return PNGF_EINVAL;
    if (cfg->refresh_k % cfg->delay_r != 0) return PNGF_EINVAL;  // refresh right after a flush
  }
  if (!(cfg->tau >= 0.0)) return PNGF_EINVAL;
  for (int p = 0; p < cfg->n_o; ++p)  // S_p = (o_p - off_p) scale_p must be invertible
    if (cfg->s_scale[2 * p] == 0.0 && cfg->s_scale[2 * p + 1] == 0.0) return PNGF_EINVAL;
  return PNGF_OK;
}

}  // namespace pngf

using namespace pngf;

extern "C" {

pngf_status pngf_workspace_size(const pngf_config* cfg, size_t* bytes) {
  pngf_status st = check_config(cfg);
  if (st != PNGF_OK) return st;
  if (!bytes) return PNGF_EINVAL;
  *bytes = make_layout(*cfg).total;
  return PNGF_OK;
}

pngf_status pngf_create(const pngf_config* cfg, const double* G_dd, const double* G_od, const double* c_d,
                        const double* c_o, const double* dv, void* workspace, size_t workspace_bytes,
                        pngf_stream stream, pngf_ctx** out) {
  if (!out) return PNGF_EINVAL;
  *out = nullptr;
  pngf_status st = check_config(cfg);
  if (st != PNGF_OK) return st;
  if (!G_dd || !G_od || !c_d || !c_o || !dv || !workspace) return PNGF_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return PNGF_EINVAL;
  for (const void* p : {(const void*)G_dd, (const void*)G_od, (const void*)c_d, (const void*)c_o, (const void*)dv})
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return PNGF_EINVAL;
  Layout L = make_layout(*cfg);
  if (workspace_bytes < L.total) return PNGF_ENOMEM;
  pngf_ctx* c = new (std::nothrow) pngf_ctx();
  if (!c) return PNGF_ENOMEM;
  c->cfg = *cfg;
  c->L = L;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->G = reinterpret_cast<const c128*>(G_dd);
  c->God = reinterpret_cast<const c128*>(G_od);
  c->cd = reinterpret_cast<const c128*>(c_d);
  c->co = reinterpret_cast<const c128*>(c_o);
  c->dv = reinterpret_cast<const c128*>(dv);
  c->ws = static_cast<char*>(workspace);
  c->obj.n_o = cfg->n_o;
  c->obj.kind = cfg->objective;
  c->obj.tau = cfg->tau;
  for (int p = 0; p < kMaxPorts; ++p) {
    c->obj.w[p] = p < cfg->n_o ? cfg->obj_weights[p] : 0.0;
    c->obj.off[p] = p < cfg->n_o ? mk(cfg->s_off[2 * p], cfg->s_off[2 * p + 1]) : mk(0.0, 0.0);
    c->obj.scale[p] = p < cfg->n_o ? mk(cfg->s_scale[2 * p], cfg->s_scale[2 * p + 1]) : mk(0.0, 0.0);
  }
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return PNGF_ECUDA;
  }
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
  if (!coop) {
    delete c;
    return PNGF_ECUDA;
  }
  c->coop_ctas = sweep_grid_size(c);
  Control* ctl = at<Control>(c, L.ctl);
  if (cudaMemsetAsync(ctl, 0, sizeof(Control), c->stream) != cudaSuccess) {
    delete c;
    return PNGF_ECUDA;
  }
  *out = c;
  return PNGF_OK;
}

pngf_status pngf_factor(pngf_ctx* c, const uint8_t* b) {
  if (!c || !b) return PNGF_EINVAL;
  if (c->cfg.precision == PNGF_PEC) {
    pngf_status st = factor_pec(c, b);
    if (st == PNGF_OK) c->factored = true;
    return st;
  }
  pngf_status st = factor_fp64(c, b);
  if (st == PNGF_OK && c->cfg.precision == PNGF_MIXED) st = mixed_after_factor(c);
  if (st == PNGF_OK) c->factored = true;
  return st;
}

pngf_status pngf_score_flips(pngf_ctx* c, const int32_t* pixels, int32_t n, double* f_new, double* o_new) {
  if (!c || n < 0 || (n > 0 && (!pixels || !f_new))) return PNGF_EINVAL;
  if (!c->factored) return PNGF_ENOTFACTORED;
  if (c->cfg.precision == PNGF_PEC) return o_new ? PNGF_EINVAL : score_flips_pec(c, pixels, n, f_new);
  return score_flips(c, pixels, n, f_new, o_new);
}

pngf_status pngf_accept_flip(pngf_ctx* c, int32_t pixel) {
  if (!c || pixel < 0 || pixel >= c->cfg.n_d) return PNGF_EINVAL;
  if (!c->factored) return PNGF_ENOTFACTORED;
  if (c->cfg.precision == PNGF_PEC) return accept_flip_pec(c, pixel);
  return c->cfg.precision == PNGF_MIXED ? accept_flip_mixed(c, pixel) : accept_flip(c, pixel);
}

pngf_status pngf_accept_flip_noalloc(pngf_ctx* c, int32_t pixel) {
  if (!c || pixel < 0 || pixel >= c->cfg.n_d) return PNGF_EINVAL;
  if (c->cfg.precision != PNGF_FP64) return PNGF_EINVAL;
  if (c->cfg.n_d > PNGF_NOALLOC_MAX_ND) return PNGF_EINVAL;
  if (!c->factored) return PNGF_ENOTFACTORED;
  return accept_flip_noalloc(c, pixel);
}

pngf_status pngf_dbs_sweep(pngf_ctx* c, int32_t n_sweeps, const int32_t* order, int32_t* trace,
                           double* trace_f, int32_t trace_cap, int64_t* counters) {
  if (!c || n_sweeps < 0 || trace_cap < 0) return PNGF_EINVAL;
  if (trace_cap > 0 && !trace && !trace_f) return PNGF_EINVAL;
  if (!c->factored) return PNGF_ENOTFACTORED;
  if (n_sweeps == 0) return PNGF_OK;
  if (c->cfg.precision == PNGF_MIXED) return run_sweep_mixed(c, n_sweeps, order, trace, trace_f, trace_cap, counters);
  if (c->cfg.precision == PNGF_PEC) return run_sweep_pec(c, n_sweeps, order, trace, trace_f, trace_cap, counters);
  return run_sweep(c, n_sweeps, order, trace, trace_f, trace_cap, counters);
}

pngf_status pngf_batch_workspace_size(int32_t n_ctx, size_t* bytes) {
  if (n_ctx < 1 || n_ctx > PNGF_BATCH_MAX_RUNS || !bytes) return PNGF_EINVAL;
  *bytes = batch_workspace_bytes(n_ctx);
  return PNGF_OK;
}

pngf_status pngf_dbs_sweep_batch(pngf_ctx* const* ctxs, int32_t n_ctx, int32_t n_sweeps,
                                 const int32_t* const* orders, int32_t* const* traces, double* const* trace_f,
                                 int32_t trace_cap, int64_t* counters, void* batch_ws, size_t batch_ws_bytes) {
  if (!ctxs || n_ctx < 1 || n_ctx > PNGF_BATCH_MAX_RUNS || n_sweeps < 0 || trace_cap < 0 || !batch_ws)
    return PNGF_EINVAL;
  if (batch_ws_bytes < batch_workspace_bytes(n_ctx)) return PNGF_ENOMEM;
  if (reinterpret_cast<uintptr_t>(batch_ws) % 256 != 0) return PNGF_EINVAL;
  const pngf_ctx* c0 = ctxs[0];
  if (!c0) return PNGF_EINVAL;
  for (int r = 0; r < n_ctx; ++r) {
    const pngf_ctx* c = ctxs[r];
    if (!c) return PNGF_EINVAL;
    if (!c->factored) return PNGF_ENOTFACTORED;
    if (c->cfg.precision != c0->cfg.precision || c->cfg.mode != c0->cfg.mode) return PNGF_EINVAL;
    if (c->cfg.precision == PNGF_PEC) return PNGF_EINVAL;
    if (c->cfg.precision == PNGF_MIXED && c->cfg.tensor_fold != c0->cfg.tensor_fold) return PNGF_EINVAL;
    if (c->cfg.n_d > PNGF_BATCH_MAX_ND || c->device != c0->device) return PNGF_EINVAL;
  }
  if (n_sweeps == 0) return PNGF_OK;
  return run_sweep_batch(ctxs, n_ctx, n_sweeps, orders, traces, trace_f, trace_cap, counters, batch_ws,
                         batch_ws_bytes);
}

pngf_status pngf_eval_ports(pngf_ctx* c, double* o_host, double* f_host) {
  if (!c) return PNGF_EINVAL;
  if (!c->factored) return PNGF_ENOTFACTORED;
  Control h;
  Control* ctl = at<Control>(c, c->L.ctl);
  if (cudaMemcpyAsync(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return PNGF_ECUDA;
  if (o_host)
    for (int p = 0; p < c->cfg.n_o; ++p) {
      o_host[2 * p] = h.o[p].x;
      o_host[2 * p + 1] = h.o[p].y;
    }
  if (f_host) *f_host = h.f;
  return h.status ? (pngf_status)h.status : PNGF_OK;
}

pngf_status pngf_get_design(pngf_ctx* c, uint8_t* b) {
  if (!c || !b) return PNGF_EINVAL;
  return cuda_status(cudaMemcpyAsync(b, at<uint8_t>(c, c->L.b), c->cfg.n_d, cudaMemcpyDeviceToDevice, c->stream));
}

pngf_status pngf_get_state(pngf_ctx* c, double* W, double* diag_W, double* e, double* T, double* o) {
  if (!c) return PNGF_EINVAL;
  if (!c->factored) return PNGF_ENOTFACTORED;
  const size_t n = c->cfg.n_d, n_o = c->cfg.n_o, cs = sizeof(c128);
  cudaStream_t s = c->stream;
  if (W) {
    if (c->cfg.precision == PNGF_MIXED) return PNGF_EINVAL;
    if (cudaMemcpy2DAsync(W, n * cs, at<c128>(c, c->L.W), (size_t)c->L.ldw * cs, n * cs, n,
                          cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return PNGF_ECUDA;
  }
  if (diag_W && cudaMemcpyAsync(diag_W, at<c128>(c, c->L.diag), n * cs, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PNGF_ECUDA;
  if (e && cudaMemcpyAsync(e, at<c128>(c, c->L.e), n * cs, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PNGF_ECUDA;
  if (T && cudaMemcpy2DAsync(T, n * cs, at<c128>(c, c->L.T), (size_t)c->L.ldt * cs, n * cs, n_o,
                             cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PNGF_ECUDA;
  if (o && cudaMemcpyAsync(o, &at<Control>(c, c->L.ctl)->o[0], n_o * cs, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PNGF_ECUDA;
  return PNGF_OK;
}

pngf_status pngf_snapshot(pngf_ctx* c) {
  if (!c) return PNGF_EINVAL;
  if (!c->factored) return PNGF_ENOTFACTORED;
  const Layout& L = c->L;

  cudaStream_t s = c->stream;
  size_t wbytes = L.snapW_bytes;
  size_t wsrc = c->cfg.precision == PNGF_MIXED ? L.Wlo_re : L.W;
  if (cudaMemcpyAsync(c->ws + L.snapW, c->ws + wsrc, wbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(c->ws + L.snapState, c->ws + L.diag, L.state_bytes, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->ws + L.snapState + L.state_bytes, c->ws + L.ctl, sizeof(Control),
                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PNGF_ECUDA;
  c->has_snapshot = true;
  return PNGF_OK;
}

pngf_status pngf_restore(pngf_ctx* c) {
  if (!c) return PNGF_EINVAL;
  if (!c->has_snapshot) return PNGF_ENOTFACTORED;
  const Layout& L = c->L;

  cudaStream_t s = c->stream;
  size_t wbytes = L.snapW_bytes;
  size_t wdst = c->cfg.precision == PNGF_MIXED ? L.Wlo_re : L.W;
  // the control block is restored from its maintained fields on (f onwards): the
  // latched status and the barrier words stay as they are
  const size_t tail = offsetof(Control, f);
  if (cudaMemcpyAsync(c->ws + wdst, c->ws + L.snapW, wbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(c->ws + L.diag, c->ws + L.snapState, L.state_bytes, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->ws + L.ctl + tail, c->ws + L.snapState + L.state_bytes + tail, sizeof(Control) - tail,
                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PNGF_ECUDA;
  return PNGF_OK;
}

pngf_status pngf_get_phase_cycles(pngf_ctx* c, int64_t* host16) {
  if (!c || !host16) return PNGF_EINVAL;
  Control* ctl = at<Control>(c, c->L.ctl);
  if (cudaMemcpyAsync(host16, ctl->phase_cycles, 16 * sizeof(long long), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return PNGF_ECUDA;
  return PNGF_OK;
}

pngf_status pngf_sync(pngf_ctx* c) {
  if (!c) return PNGF_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return PNGF_ECUDA;
  Control* ctl = at<Control>(c, c->L.ctl);
  int st = 0;
  if (cudaMemcpy(&st, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PNGF_ECUDA;
  if (st) {
    int zero = 0;
    if (cudaMemcpy(&ctl->status, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return PNGF_ECUDA;
  }
  return (pngf_status)st;
}

pngf_status pngf_tiles_workspace_size(int32_t n_sys, int32_t n_d, int32_t n_tiles, int32_t tile_m, size_t* bytes) {
  if (n_sys < 1 || n_sys > PNGF_TILES_MAX_SYSTEMS || n_d < 1 || n_d > 32768 || n_tiles < 1 ||
      tile_m < 1 || tile_m > PNGF_TILE_MAX || !bytes)
    return PNGF_EINVAL;
  *bytes = tiles_workspace_bytes(n_sys, n_d, n_tiles, tile_m);
  return PNGF_OK;
}

// the systems of one tile search: FP64, factored, one device, one size, objective and mode
static pngf_status check_tile_call(pngf_ctx* const* ctxs, int32_t n_sys, int32_t combine, const int32_t* tiles,
                                   int32_t n_tiles, int32_t tile_m, void* ws, size_t ws_bytes) {
  if (!ctxs || n_sys < 1 || n_sys > PNGF_TILES_MAX_SYSTEMS || !tiles || n_tiles < 1 || tile_m < 1 ||
      tile_m > PNGF_TILE_MAX || !ws)
    return PNGF_EINVAL;
  if (combine != PNGF_COMBINE_MEAN && combine != PNGF_COMBINE_WORST) return PNGF_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return PNGF_EINVAL;
  const pngf_ctx* c0 = ctxs[0];
  if (!c0) return PNGF_EINVAL;
  if (ws_bytes < tiles_workspace_bytes(n_sys, c0->cfg.n_d, n_tiles, tile_m)) return PNGF_ENOMEM;
  for (int s = 0; s < n_sys; ++s) {
    const pngf_ctx* c = ctxs[s];
    if (!c) return PNGF_EINVAL;
    if (!c->factored) return PNGF_ENOTFACTORED;
    if (c->cfg.precision != PNGF_FP64 || c->cfg.n_d != c0->cfg.n_d || c->device != c0->device ||
        c->cfg.objective != c0->cfg.objective || c->cfg.mode != c0->cfg.mode)
      return PNGF_EINVAL;
  }
  return PNGF_OK;
}

pngf_status pngf_dbs_sweep_tiles(pngf_ctx* const* ctxs, int32_t n_sys, int32_t combine, const int32_t* tiles,
                                 int32_t n_tiles, int32_t tile_m, int32_t n_sweeps, const int32_t* order,
                                 int32_t* trace, double* trace_f, int32_t trace_cap, int64_t* counters, void* ws,
                                 size_t ws_bytes) {
  pngf_status st = check_tile_call(ctxs, n_sys, combine, tiles, n_tiles, tile_m, ws, ws_bytes);
  if (st != PNGF_OK) return st;
  if (n_sweeps < 0 || trace_cap < 0 || (trace_cap > 0 && !trace && !trace_f)) return PNGF_EINVAL;
  if (n_sweeps == 0) return PNGF_OK;
  return run_sweep_tiles(ctxs, n_sys, combine, tiles, n_tiles, tile_m, n_sweeps, order, -1, trace, trace_f,
                         trace_cap, counters, ws);
}

pngf_status pngf_score_tiles(pngf_ctx* const* ctxs, int32_t n_sys, int32_t combine, const int32_t* tiles,
                             int32_t n_tiles, int32_t tile_m, const int32_t* list, int32_t count, double* F,
                             double* f_sys, void* ws, size_t ws_bytes) {
  pngf_status st = check_tile_call(ctxs, n_sys, combine, tiles, n_tiles, tile_m, ws, ws_bytes);
  if (st != PNGF_OK) return st;
  if (count < 0 || (count > 0 && (!list || !F))) return PNGF_EINVAL;
  return score_tiles(ctxs, n_sys, combine, tiles, n_tiles, tile_m, list, count, F, f_sys, ws);
}

pngf_status pngf_accept_tile(pngf_ctx* const* ctxs, int32_t n_sys, int32_t combine, const int32_t* tiles,
                             int32_t n_tiles, int32_t tile_m, int32_t tile, void* ws, size_t ws_bytes) {
  pngf_status st = check_tile_call(ctxs, n_sys, combine, tiles, n_tiles, tile_m, ws, ws_bytes);
  if (st != PNGF_OK) return st;
  if (tile < 0 || tile >= n_tiles) return PNGF_EINVAL;
  return run_sweep_tiles(ctxs, n_sys, combine, tiles, n_tiles, tile_m, 1, nullptr, tile, nullptr, nullptr, 0,
                         nullptr, ws);
}

pngf_status pngf_set_launch(pngf_ctx* c, int32_t n_ctas, int32_t tensor_fold) {
  if (!c || n_ctas < 0 || (tensor_fold != 0 && tensor_fold != 1)) return PNGF_EINVAL;
  if (tensor_fold && c->cfg.precision != PNGF_MIXED) return PNGF_EINVAL;
  c->cfg.n_ctas = n_ctas;
  c->cfg.tensor_fold = tensor_fold;
  c->coop_ctas = sweep_grid_size(c);
  return PNGF_OK;
}

pngf_status pngf_gradient(pngf_ctx* c, double* grad, double* dodrho) {
  if (!c || !grad) return PNGF_EINVAL;
  if (!c->factored) return PNGF_ENOTFACTORED;
  if (c->cfg.precision == PNGF_PEC) return PNGF_EINVAL;
  return gradient(c, grad, dodrho);
}

pngf_status pngf_set_wait_limit(pngf_ctx* c, int32_t wait_log2, int32_t hold_cta) {
  if (!c) return PNGF_EINVAL;
  if (wait_log2 != 0 && (wait_log2 < 8 || wait_log2 > 30)) return PNGF_EINVAL;
  if (hold_cta < -1 || hold_cta >= c->coop_ctas) return PNGF_EINVAL;
  return set_wait_limit(c, wait_log2 ? (1ull << wait_log2) : 0ull, hold_cta + 1);
}

pngf_status pngf_get_since_refresh(pngf_ctx* c, int32_t* since_refresh) {
  if (!c || !since_refresh) return PNGF_EINVAL;
  if (!c->factored) return PNGF_ENOTFACTORED;
  Control* ctl = at<Control>(c, c->L.ctl);
  if (cudaMemcpyAsync(since_refresh, &ctl->since_refresh, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return PNGF_ECUDA;
  return PNGF_OK;
}

pngf_status pngf_set_state(pngf_ctx* c, const uint8_t* b, const double* W, const double* diag_W, const double* e,
                           const double* T, const double* o, int32_t since_refresh) {
  if (!c || !diag_W || !e || !T || !o || since_refresh < 0) return PNGF_EINVAL;
  if (!c->factored) return PNGF_ENOTFACTORED;
  if (c->cfg.precision == PNGF_PEC) return PNGF_EINVAL;
  const bool fp64 = c->cfg.precision == PNGF_FP64;
  if (fp64 ? (!W || !b) : (W || b)) return PNGF_EINVAL;
  if (!fp64 && c->cfg.refresh_k > 0 && since_refresh >= c->cfg.refresh_k) return PNGF_EINVAL;
  const size_t n = c->cfg.n_d, n_o = c->cfg.n_o, cs = sizeof(c128);
  cudaStream_t s = c->stream;
  if (fp64) {
    if (cudaMemcpy2DAsync(at<c128>(c, c->L.W), (size_t)c->L.ldw * cs, W, n * cs, n * cs, n,
                          cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(at<uint8_t>(c, c->L.b), b, n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return PNGF_ECUDA;
  }
  if (cudaMemcpyAsync(at<c128>(c, c->L.diag), diag_W, n * cs, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(at<c128>(c, c->L.e), e, n * cs, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpy2DAsync(at<c128>(c, c->L.T), (size_t)c->L.ldt * cs, T, n * cs, n * cs, n_o,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(&at<Control>(c, c->L.ctl)->o[0], o, n_o * cs, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PNGF_ECUDA;
  return import_finish(c, since_refresh);
}

const char* pngf_status_string(pngf_status s) {
  switch (s) {
    case PNGF_OK: return "ok";
    case PNGF_EINVAL: return "invalid argument";
    case PNGF_ENOMEM: return "workspace too small";
    case PNGF_ECUDA: return "CUDA runtime error";
    case PNGF_ESINGULAR: return "singular system matrix (zero pivot)";
    case PNGF_ENOTFACTORED: return "not factored";
    case PNGF_ETIMEOUT: return "device wait timed out";
    case PNGF_ENUMERIC: return "non-finite value";
    case PNGF_ECAPACITY: return "trace buffer full";
    case PNGF_EACCURACY: return "mixed precision lost accuracy (ill-conditioned system)";
  }
  return "unknown status";
}

void pngf_destroy(pngf_ctx* c) { delete c; }

}  // extern "C"
