// Direct binary search on the device (FP64 path).
//
// Per kept flip of pixel k (section "Low-rank update evaluation", Eqs. 9-14 in
// the field form of Supplementary Note 4; the cost split of Supplementary
// Note 3):
//   score   for every remaining pixel j: delta_j = +-dv_j, d_j = 1 - delta_j W_jj,
//           alpha_j = delta_j / d_j, o^(j) = o + alpha_j e_j T[:,j], f^(j)
//   select  FIRST: earliest visiting position with gain > tau*max(|f|,1e-30);
//           BEST: largest gain, ties -> lowest pixel index
//   accept  c = W[:,k] (= W[k,:]^T, W is complex symmetric),
//           W += alpha c c^T (upper triangle), T += alpha T[:,k] c^T,
//           e += alpha e_k c, o = o^(k), v_k, b_k flipped
//   refresh every refresh_k kept flips: one FP64 iterative-refinement step
//           of e and T against G (residuals r = c_d - M e, R = G_od - T M^T,
//           corrections (I + W V) r and R (I + V W)), then o = c_o + G_od V e
//
// One cooperative launch runs the whole search.  Pixels are split into
// contiguous chunks, one per CTA; the packed upper triangle of W is split
// into equal element ranges, one per CTA.  Grid-wide barriers are a counter
// plus generation word with a bounded spin: a barrier that waits longer than
// the spin limit latches PNGF_ETIMEOUT and every CTA returns.
#include <cstdio>
#include <mutex>

#include "rank1.cuh"

namespace pngf {
namespace {

// ---------------------------------------------------------------- persistent DBS
__global__ void __launch_bounds__(kThreads) dbs_fp64_kernel(SweepArgs a) {
  extern __shared__ int act_smem[];  // n entries: active-pixel list of the refresh
  const int P = gridDim.x, cta = blockIdx.x;
  const int n = a.n;
  const int pb = (int)((long long)n * cta / P), pe = (int)((long long)n * (cta + 1) / P);
  const long long E = (long long)n * (n + 1) / 2;
  const long long eb = E * cta / P, ee = E * (cta + 1) / P;
  Control* ctl = a.ctl;
  hold_if_asked(ctl);
  // search state shared by the CTA (identical in every CTA: each one derives it
  // from the same data in the same order)
  __shared__ c128 s_o[kMaxPorts];
  __shared__ double s_f;
  __shared__ Pivot s_pv;
  __shared__ int s_k, s_pos;
  __shared__ ObjParams s_op;
  if (threadIdx.x == 0) {
    s_op = a.op;
    FOR_PORTS(p, a.n_o) s_o[p] = ctl->o[p];
    s_f = ctl->f;
  }
  __syncthreads();
  long long n_acc = 0, n_evals = 0, n_refresh = 0, sum_active = 0;
  int sweeps_done = 0, converged = 0, status = PNGF_OK;
  // per-phase SM-cycle accounting of CTA 0 (thread 0 sees every phase boundary)
  const bool timer = (cta == 0 && threadIdx.x == 0);
  long long ph[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  long long t_last = clock64(), t_begin = t_last;
  auto tick = [&](int phase) {
    if (timer) {
      long long now = clock64();
      ph[phase] += now - t_last;
      t_last = now;
    }
  };
  int since_refresh = ctl->since_refresh;
  int s = 0, t = 0, acc_in_sweep = 0, slot = 0, rd = 0;
  bool failed = false;

  // inverse permutation of the sweep's visiting order; an entry outside
  // [0, n) is rejected (latched PNGF_EINVAL, the search stops)
  auto setup_sweep = [&](int sw) {
    if (a.order)
      for (int q = pb + threadIdx.x; q < pe; q += blockDim.x) {
        int px = a.order[(size_t)sw * n + q];
        if ((unsigned)px < (unsigned)n) a.pos_of[px] = q;
        else latch_status(ctl, PNGF_EINVAL);
      }
  };
  if (a.mode == PNGF_FIRST_IMPROVEMENT && a.order) {
    setup_sweep(0);
    if (!grid_sync(ctl)) failed = true;
    else if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) status = PNGF_EINVAL;
  }
  const long long max_steps = a.n_sweeps;  // BEST mode: one kept flip per step
  while (!failed && status != PNGF_EINVAL) {
    const double f = s_f;
    const double thr = accept_threshold(s_op, f);
    // ---- score own pixels and reduce to this CTA's candidate
    if (a.mode == PNGF_FIRST_IMPROVEMENT) {
      long long best = LLONG_MAX;
      for (int j = pb + threadIdx.x; j < pe; j += blockDim.x) {
        int pos = a.order ? a.pos_of[j] : j;
        if (pos < t) continue;
        double fn;
        if (!score_pixel(a, s_op, j, s_o, fn, nullptr)) continue;
        if (gain_of(s_op, fn, f) - thr > 0.0 && pos < best) best = pos;
      }
      best = block_min_ll(best);
      if (threadIdx.x == 0) sel_offer(ctl, rd, best, cta);
      tick(0);
    } else {
      double g = -INFINITY;
      int pix = INT_MAX;
      for (int j = pb + threadIdx.x; j < pe; j += blockDim.x) {
        double fn;
        if (!score_pixel(a, s_op, j, s_o, fn, nullptr)) continue;
        double gg = gain_of(s_op, fn, f);
        if (better(gg, j, g, pix)) { g = gg; pix = j; }
      }
      block_best(g, pix);
      if (threadIdx.x == 0) {
        a.part_gain[slot * P + cta] = g;
        a.part_key[slot * P + cta] = pix;
      }
      tick(0);
    }
    if (!grid_sync(ctl)) { failed = true; break; }
    tick(1);
    // ---- warp 0 of every CTA reduces the partials (a fixed shuffle order, so
    //      every CTA obtains the same result); lane 0 then forms the pivot
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      int k = -1, pos_k = -1;
      if (a.mode == PNGF_FIRST_IMPROVEMENT) {
        unsigned long long key = sel_read(ctl, rd);
        if (key != ~0ull) {
          pos_k = (int)(key >> 10);
          k = a.order ? a.order[(size_t)s * n + pos_k] : pos_k;
          if ((unsigned)k >= (unsigned)n) k = -2;  // invalid order entry
        }
      } else {
        double g = -INFINITY;
        int pix = INT_MAX;
        for (int q = lane; q < P; q += 32) {
          double gg = a.part_gain[slot * P + q];
          int pp = (int)a.part_key[slot * P + q];
          if (better(gg, pp, g, pix)) { g = gg; pix = pp; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          double og = __shfl_xor_sync(0xffffffffu, g, off);
          int op = __shfl_xor_sync(0xffffffffu, pix, off);
          if (better(og, op, g, pix)) { g = og; pix = op; }
        }
        if (pix != INT_MAX && g - thr > 0.0) k = pix;
        pos_k = 0;
      }
      if (lane == 0) {
        s_k = k;
        s_pos = pos_k;
        if (k >= 0) {
          // pivot of the kept flip and the new ports / objective (Eq. 14)
          make_pivot(a, k, s_pv);
          FOR_PORTS(p, a.n_o) s_o[p] = cfma(s_pv.coef, s_pv.Tk[p], s_o[p]);
          s_f = objective_of(s_op, s_o);
        }
      }
    }
    __syncthreads();
    slot ^= 1;
    ++rd;
    const int k = s_k, pos_k = s_pos;
    if (k == -2) {  // invalid visiting-order entry
      status = PNGF_EINVAL;
      break;
    }
    if (k < 0) {
      // nothing improves in the rest of this sweep (FIRST) / anywhere (BEST)
      if (a.mode == PNGF_FIRST_IMPROVEMENT) {
        n_evals += n - t;
        ++sweeps_done;
        if (acc_in_sweep == 0) { converged = 1; break; }
        ++s;
        if (s >= a.n_sweeps) break;
        t = 0;
        acc_in_sweep = 0;
        if (a.order) {
          setup_sweep(s);
          if (!grid_sync(ctl)) { failed = true; break; }
          if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) { status = PNGF_EINVAL; break; }
        }
        tick(6);
        continue;
      } else {
        n_evals += n;
        ++sweeps_done;
        converged = 1;
        break;
      }
    }
    // ---- accept pixel k
    if (!isfinite(s_f)) status = PNGF_ENUMERIC;
    if (a.mode == PNGF_FIRST_IMPROVEMENT) {
      n_evals += pos_k - t + 1;
      t = pos_k + 1;
    } else {
      n_evals += n;
      ++sweeps_done;
    }
    ++acc_in_sweep;
    if (cta == 0 && threadIdx.x == 0) {
      if (n_acc < a.trace_cap) {
        if (a.trace) {
          int32_t* tr = a.trace + 4 * n_acc;
          tr[0] = a.mode == PNGF_FIRST_IMPROVEMENT ? s : (int)n_acc;
          tr[1] = pos_k;
          tr[2] = k;
          tr[3] = 0;
        }
        if (a.trace_f) a.trace_f[n_acc] = s_f;
      } else if (status == PNGF_OK) {
        status = PNGF_ECAPACITY;
      }
    }
    ++n_acc;
    // c = W[:,k] and alpha c (block 3 of the refresh scratch, free between refreshes)
    gather_column_ac(a, k, s_pv.alpha, rvec(a, 3, 0), pb, pe);
    tick(2);
    if (!grid_sync(ctl)) { failed = true; break; }
    tick(3);
    update_state(a, s_pv, pb, pe);
    rank1_upper_ac(a.W, n, a.ldw, rvec(a, 3, 0), a.cbuf, eb, ee);
    __syncthreads();
    tick(4);
    ++since_refresh;
    if (a.refresh_k > 0 && since_refresh >= a.refresh_k) {
      since_refresh = 0;
      ++n_refresh;
      if (!grid_sync(ctl)) { failed = true; break; }
      tick(5);
      refresh_x(a, pb, pe);
      if (!grid_sync(ctl)) { failed = true; break; }
      tick(8);
      const int m_act = refresh_residual(a, pb, pe, act_smem);
      sum_active += m_act;
      const int t_end = count_below(act_smem, m_act, pe - 1);
      if (!grid_sync(ctl)) { failed = true; break; }
      tick(9);
      correct_strips<false>(a, pb, pe, a.actg, t_end, reinterpret_cast<float*>(act_smem),
                            (int)dynamic_smem_bytes());
      if (!grid_sync(ctl)) { failed = true; break; }
      tick(10);
      ports_partial(a, pb, pe);
      if (!grid_sync(ctl)) { failed = true; break; }
      tick(11);
      ports_total(a, s_o);
      if (threadIdx.x == 0) s_f = objective_of(s_op, s_o);
      __syncthreads();
      // no CTA rewrites opart before the next refresh, many barriers later
      tick(5);
    }
    if (status == PNGF_ENUMERIC) break;
    if (a.mode == PNGF_BEST_IMPROVEMENT && n_acc >= max_steps) break;
    if (a.mode == PNGF_FIRST_IMPROVEMENT && t >= n) {
      // the sweep ended on an accepted flip at its last position
      ++sweeps_done;
      ++s;
      if (s >= a.n_sweeps) break;
      t = 0;
      acc_in_sweep = 0;
      if (a.order) {
        if (!grid_sync(ctl)) { failed = true; break; }
        setup_sweep(s);
        if (!grid_sync(ctl)) { failed = true; break; }
        if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) { status = PNGF_EINVAL; break; }
      }
    }
  }
  if (cta == 0 && threadIdx.x == 0) {
    if (failed) status = PNGF_ETIMEOUT;
    FOR_PORTS(p, a.n_o) ctl->o[p] = s_o[p];
    ctl->f = s_f;
    ctl->since_refresh = since_refresh;
    ctl->n_acc_total += (int)n_acc;
    ctl->counters[0] = n_acc;
    ctl->counters[1] = n_evals;
    ctl->counters[2] = sweeps_done;
    ctl->counters[3] = converged;
    ctl->counters[4] = n_refresh;
    ctl->counters[5] = 0;
    ctl->counters[6] = status;
    ctl->counters[7] = sum_active;
    ph[7] = clock64() - t_begin;
    for (int q = 0; q < 16; ++q) ctl->phase_cycles[q] = ph[q];
    if (a.counters)
      for (int q = 0; q < 8; ++q) a.counters[q] = ctl->counters[q];
    if (status == PNGF_ENUMERIC || status == PNGF_ETIMEOUT || status == PNGF_EINVAL) latch_status(ctl, status);
  }
}

// ---------------------------------------------------------------- single calls
__global__ void score_kernel(SweepArgs a, const int32_t* __restrict__ pixels, int m,
                             double* __restrict__ f_new, c128* __restrict__ o_new) {
  __shared__ ObjParams s_op;
  __shared__ c128 o[kMaxPorts];
  if (threadIdx.x == 0) {
    s_op = a.op;
    FOR_PORTS(p, a.n_o) o[p] = a.ctl->o[p];
  }
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    int j = pixels[i];
    double fn = NAN;
    c128 on[kMaxPorts];
    bool ok = (j >= 0 && j < a.n) && score_pixel(a, s_op, j, o, fn, on);
    f_new[i] = ok ? fn : NAN;
    if (o_new) {
      FOR_PORTS(p, a.n_o) o_new[(size_t)i * a.n_o + p] = ok ? on[p] : mk(NAN, NAN);
    }
  }
}

// one CTA: pivot of pixel k, new o and f, column copy into cbuf, pivot record
struct PivotRecord {
  Pivot pv;
};

__global__ void accept_pivot_kernel(SweepArgs a, int k, PivotRecord* rec) {
  if (threadIdx.x == 0) {
    Pivot pv;
    make_pivot(a, k, pv);
    rec->pv = pv;
    c128 o[kMaxPorts];
    FOR_PORTS(p, a.n_o) o[p] = cfma(pv.coef, pv.Tk[p], a.ctl->o[p]);
    FOR_PORTS(p, a.n_o) a.ctl->o[p] = o[p];
    a.ctl->f = objective_of(a.op, o);
    a.ctl->n_acc_total += 1;
  }
}

__global__ void accept_gather_kernel(SweepArgs a, int k) {
  int per = (a.n + gridDim.x - 1) / gridDim.x;
  int pb = blockIdx.x * per, pe = min(a.n, pb + per);
  gather_column(a, k, pb, pe);
}

__global__ void __launch_bounds__(kThreads) accept_update_kernel(SweepArgs a, const PivotRecord* rec) {
  const int P = gridDim.x, cta = blockIdx.x, n = a.n;
  const int pb = (int)((long long)n * cta / P), pe = (int)((long long)n * (cta + 1) / P);
  const long long E = (long long)n * (n + 1) / 2;
  Pivot pv = rec->pv;
  update_state(a, pv, pb, pe);
  rank1_upper(a.W, n, a.ldw, a.cbuf, pv.alpha, E * cta / P, E * (cta + 1) / P);
}

__global__ void set_wait_kernel(Control* ctl, unsigned long long polls, int hold_plus1) {
  ctl->spin_limit = polls;
  ctl->hold_cta = hold_plus1;
  ctl->hold_flag = 0;
}

// after an imported state: v from b, f from o, the refresh phase
__global__ void import_finish_kernel(SweepArgs a, int since_refresh) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += gridDim.x * blockDim.x)
    a.v[j] = a.b[j] ? a.dv[j] : mk(0.0, 0.0);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl->f = objective_of(a.op, a.ctl->o);
    a.ctl->since_refresh = since_refresh;
  }
}

}  // namespace

pngf_status set_wait_limit(pngf_ctx* c, unsigned long long polls, int hold_plus1) {
  set_wait_kernel<<<1, 1, 0, c->stream>>>(at<Control>(c, c->L.ctl), polls, hold_plus1);
  return cuda_status(cudaGetLastError());
}

pngf_status import_finish(pngf_ctx* c, int since_refresh) {
  SweepArgs a = make_args(c);
  int blocks = (c->cfg.n_d + 255) / 256;
  if (blocks > c->n_sm) blocks = c->n_sm;
  import_finish_kernel<<<blocks, 256, 0, c->stream>>>(a, since_refresh);
  return cuda_status(cudaGetLastError());
}

// active-pixel list of the refresh residual, then the staging of the correction
static size_t fp64_smem(int n) {
  const size_t act = (size_t)n * sizeof(int), ct = (size_t)110 * 1024;  // room to stage x2 of n_d = 4096 at once
  return act > ct ? act : ct;
}

int sweep_grid_size(pngf_ctx* c) {
  static bool attr = false;
  if (!attr) {  // room for the largest region (n_d <= 32768)
    cudaFuncSetAttribute(dbs_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fp64_smem(32768));
    attr = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dbs_fp64_kernel, kThreads, fp64_smem(c->cfg.n_d));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;
  int g = c->n_sm * per_sm;
  if (c->cfg.n_ctas > 0 && c->cfg.n_ctas < g) g = c->cfg.n_ctas;
  if (g > c->L.n_part) g = c->L.n_part;
  return g;
}

pngf_status run_sweep(pngf_ctx* c, int n_sweeps, const int32_t* order, int32_t* trace,
                      double* trace_f, int32_t trace_cap, int64_t* counters) {
  SweepArgs a = make_args(c);
  a.n_sweeps = n_sweeps;
  a.order = order;
  a.trace = trace;
  a.trace_f = trace_f;
  a.trace_cap = trace_cap;
  a.counters = counters;
  Control* ctl = a.ctl;
  // reset the barrier words (a previous launch that timed out may have left them set)
  cudaError_t err = cudaMemsetAsync(&ctl->bar_count, 0, 2 * sizeof(unsigned), c->stream);
  if (err != cudaSuccess) return PNGF_ECUDA;
  err = cudaMemsetAsync(&ctl->sel[0], 0xff, sizeof(ctl->sel), c->stream);
  if (err != cudaSuccess) return PNGF_ECUDA;
  int grid = c->coop_ctas;
  void* params[] = {&a};
  err = cudaLaunchCooperativeKernel((const void*)dbs_fp64_kernel, dim3(grid), dim3(kThreads), params,
                                    fp64_smem(c->cfg.n_d), c->stream);
  return cuda_status(err);
}

pngf_status score_flips(pngf_ctx* c, const int32_t* pixels, int m, double* f_new, double* o_new) {
  if (m <= 0) return PNGF_OK;
  SweepArgs a = make_args(c);
  int blocks = (m + 255) / 256;
  if (blocks > 4 * c->n_sm) blocks = 4 * c->n_sm;
  score_kernel<<<blocks, 256, 0, c->stream>>>(a, pixels, m, f_new, reinterpret_cast<c128*>(o_new));
  return cuda_status(cudaGetLastError());
}

pngf_status accept_flip(pngf_ctx* c, int pixel) {
  SweepArgs a = make_args(c);
  PivotRecord* rec = reinterpret_cast<PivotRecord*>(a.rbuf);  // scratch
  accept_pivot_kernel<<<1, 32, 0, c->stream>>>(a, pixel, rec);
  accept_gather_kernel<<<c->n_sm, 256, 0, c->stream>>>(a, pixel);
  accept_update_kernel<<<c->n_sm * 2, kThreads, 0, c->stream>>>(a, rec);
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------- accept without workspace scratch
// Scratch of the kept-flip update (the pivot record and the gathered column c)
// in a fixed device array instead of the caller's workspace, for callers that
// must not allocate device memory at all.  Every GPU that loads the library
// holds this array until the process exits.
constexpr int kNoAllocRecordBytes = 256;
static_assert(sizeof(PivotRecord) <= kNoAllocRecordBytes, "pivot record slot");
static __device__ __align__(256) unsigned char g_accept_scratch[kNoAllocRecordBytes +
                                                               PNGF_NOALLOC_MAX_ND * sizeof(c128)];

constexpr int kMaxDevices = 64;
static void* g_accept_scratch_ptr[kMaxDevices];
static std::mutex g_accept_scratch_mu;

// Device address of the array on the current device; resolved once per device.
static pngf_status accept_scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return PNGF_EINVAL;
  std::lock_guard<std::mutex> lock(g_accept_scratch_mu);
  if (!g_accept_scratch_ptr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_accept_scratch) != cudaSuccess || !p) return PNGF_ECUDA;
    g_accept_scratch_ptr[device] = p;
  }
  *out = g_accept_scratch_ptr[device];
  return PNGF_OK;
}

pngf_status accept_flip_noalloc(pngf_ctx* c, int pixel) {
  if (c->cfg.n_d > PNGF_NOALLOC_MAX_ND) return PNGF_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PNGF_ECUDA;
  if (dev != c->device) return PNGF_EINVAL;
  void* base = nullptr;
  pngf_status st = accept_scratch_address(dev, &base);
  if (st != PNGF_OK) return st;
  SweepArgs a = make_args(c);
  PivotRecord* rec = static_cast<PivotRecord*>(base);
  a.cbuf = reinterpret_cast<c128*>(static_cast<unsigned char*>(base) + kNoAllocRecordBytes);
  accept_pivot_kernel<<<1, 32, 0, c->stream>>>(a, pixel, rec);
  accept_gather_kernel<<<c->n_sm, 256, 0, c->stream>>>(a, pixel);
  accept_update_kernel<<<c->n_sm * 2, kThreads, 0, c->stream>>>(a, rec);
  return cuda_status(cudaGetLastError());
}

}  // namespace pngf
