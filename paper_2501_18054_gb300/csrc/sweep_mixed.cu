// Direct binary search on the device, mixed-precision path.
//
// The maintained inverse W = M^-1 G (the paper's C~^-1, Supplementary Note 4)
// is kept as a planar FP32 copy W_lo plus a delayed FP64 rank-r correction:
//   W = W_lo + sum_{i<r} alpha_i x_i x_i^T,   x_i = column of W at kept flip i.
// Everything that decides a flip stays FP64: diag(W), e, T, o, the
// Sherman-Morrison denominators d_k and alpha (Eqs. 9 and 14).  Per kept flip
// of pixel k only the column c = W[:,k] is needed:
//   c_j = W_lo(k, j) + sum_{i<r} (alpha_i x_i[k]) x_i[j]      (FP32 arithmetic)
// which updates diag(W), e and T in FP64 and is appended to the delayed set.
// On GB300 the FP64 pipe retires 2 DFMA per clock per SM (1/64 of FP32), so
// everything that only has to be FP32-accurate runs on the FP32 pipe.
// Every R kept flips the delayed set is folded into W_lo with one rank-R
// product over the upper triangle (the paper's O(N_opt^2) update of
// Supplementary Note 3, done once per R flips), and every refresh_k flips e
// and T are refined in FP64 against G.
//
// Each CTA publishes its best candidate together with the pixel state the
// pivot needs, so one grid barrier per kept flip suffices: nobody reads the
// state arrays of the chosen pixel while its owner updates them.
#include <cstdio>

#include "flush_tc.cuh"

namespace pngf {
namespace {

// ---------------------------------------------------------------- persistent mixed DBS
__global__ void __launch_bounds__(kThreads) dbs_mixed_kernel(SweepArgs a) {
  extern __shared__ float dyn_smem[];
  const int P = gridDim.x, cta = blockIdx.x;
  const int n = a.n;
  const int pb = (int)((long long)n * cta / P), pe = (int)((long long)n * (cta + 1) / P);
  Control* ctl = a.ctl;
  __shared__ c128 s_o[kMaxPorts];
  __shared__ double s_f;
  __shared__ Pivot s_pv;
  __shared__ int s_k, s_pos;
  __shared__ ObjParams s_op;
  __shared__ float2 s_beta[kMaxDelay];
  if (threadIdx.x == 0) {
    s_op = a.op;
    FOR_PORTS(p, a.n_o) s_o[p] = ctl->o[p];
    s_f = ctl->f;
  }
  __syncthreads();
  long long n_acc = 0, n_evals = 0, n_refresh = 0, n_flush = 0;
  int sweeps_done = 0, converged = 0, status = PNGF_OK;
  int since_refresh = ctl->since_refresh;
  int r = ctl->r_delay;
  int s = 0, t = 0, acc_in_sweep = 0, slot = 0, rd = 0;
  bool failed = false;
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
  auto setup_sweep = [&](int sw) {
    if (a.order)
      for (int q = pb + threadIdx.x; q < pe; q += blockDim.x) {
        int px = a.order[(size_t)sw * n + q];
        if ((unsigned)px < (unsigned)n) a.pos_of[px] = q;
        else latch_status(ctl, PNGF_EINVAL);
      }
  };
  // tensor-core fold: warp 0 holds TC_TMEM_COLS columns of tensor memory for the whole search
  __shared__ __align__(8) unsigned long long s_mb_load, s_mb_mma;
  __shared__ unsigned s_tmem;
  TcState tcs;
  tcs.tmem = 0;
  tcs.ph_load = tcs.ph_mma = 0;
  if (a.tensor_fold) {
    tc_mbar_init(&s_mb_load, &s_mb_mma);
    tc_alloc(&s_tmem);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    tcs.tmem = s_tmem;
    tcs.mb_load = (unsigned)__cvta_generic_to_shared(&s_mb_load);
    tcs.mb_mma = (unsigned)__cvta_generic_to_shared(&s_mb_mma);
  }
  auto flush = [&]() -> bool {
    if (!grid_sync(ctl)) return false;
    if (a.tensor_fold) {
      tc_prepare(a, r, a.tcimgA, a.tcimgB, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                 (long long)gridDim.x * blockDim.x);
      if (!grid_sync(ctl)) return false;
      if (!tc_fold_tiles(a, r, a.tcimgA, a.tcimgB, reinterpret_cast<unsigned char*>(dyn_smem), tcs, blockIdx.x,
                         gridDim.x)) {
        if (threadIdx.x == 0) latch_status(ctl, PNGF_ETIMEOUT);
        return false;
      }
    } else {
      flush_tiles(a, r, dyn_smem, blockIdx.x, gridDim.x);
    }
    if (!grid_sync(ctl)) return false;
    r = 0;
    ++n_flush;
    return true;
  };
  if (a.mode == PNGF_FIRST_IMPROVEMENT && a.order) {
    setup_sweep(0);
    if (!grid_sync(ctl)) failed = true;
    else if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) status = PNGF_EINVAL;
  }
  const long long max_steps = a.n_sweeps;
  while (!failed && status != PNGF_EINVAL) {
    const double f = s_f;
    const double thr = accept_threshold(s_op, f);
    // ---- score own pixels; the CTA's best candidate and its state go to a record
    {
      long long best = LLONG_MAX;
      double g = -INFINITY;
      int pix = INT_MAX;
      c128 b_alpha = mk(0.0, 0.0), b_coef = b_alpha;
      for (int j = pb + threadIdx.x; j < pe; j += blockDim.x) {
        double fn;
        c128 al, co;
        if (a.mode == PNGF_FIRST_IMPROVEMENT) {
          int pos = a.order ? a.pos_of[j] : j;
          if (pos < t) continue;
          if (!score_pixel(a, s_op, j, s_o, fn, nullptr, &al, &co)) continue;
          if (gain_of(s_op, fn, f) - thr > 0.0 && pos < best) {
            best = pos;
            pix = j;
            b_alpha = al;
            b_coef = co;
          }
        } else {
          if (!score_pixel(a, s_op, j, s_o, fn, nullptr, &al, &co)) continue;
          double gg = gain_of(s_op, fn, f);
          if (better(gg, j, g, pix)) {
            g = gg;
            pix = j;
            b_alpha = al;
            b_coef = co;
          }
        }
      }
      CandRecord* rc = rec_at(a, slot, cta);
      if (a.mode == PNGF_FIRST_IMPROVEMENT) {
        long long bmin = block_min_ll(best);
        if (threadIdx.x == 0) sel_offer(ctl, rd, bmin, cta);
        if (bmin == LLONG_MAX) {
          if (threadIdx.x == 0) rc->key = LLONG_MAX;
        } else if (best == bmin) {
          fill_record(a, rc, pix, best, 0.0, b_alpha, b_coef);
        }
      } else {
        double gb = g;
        int pb2 = pix;
        block_best(gb, pb2);
        if (pb2 == INT_MAX) {
          if (threadIdx.x == 0) { rc->key = LLONG_MAX; rc->gain = -INFINITY; rc->pixel = INT_MAX; }
        } else if (pix == pb2) {
          fill_record(a, rc, pix, 0, gb, b_alpha, b_coef);
        }
      }
    }
    tick(0);
    if (!grid_sync(ctl)) { failed = true; break; }
    tick(1);
    // ---- warp 0 picks the winning record; lane 0 forms the pivot while the
    //      other lanes already gather beta_i = alpha_i x_i[k] (FIRST mode: k is
    //      known from the selection cell before the record arrives)
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      int win = -1, k_pre = -1;
      if (a.mode == PNGF_FIRST_IMPROVEMENT) {
        unsigned long long key = sel_read(ctl, rd);
        if (key != ~0ull) {
          win = (int)(key & 1023u);
          int pos = (int)(key >> 10);
          k_pre = a.order ? a.order[(size_t)s * n + pos] : pos;
          if ((unsigned)k_pre >= (unsigned)n) win = -2;
          if ((unsigned)k_pre < (unsigned)n) {
            for (int i = lane; i < r; i += 32) {
              c128 al = a.xa[i];
              float2 x = a.X[(size_t)k_pre * a.R + i];
              float ax = (float)al.x, ay = (float)al.y;
              s_beta[i] = make_float2(fmaf(ax, x.x, -ay * x.y), fmaf(ax, x.y, ay * x.x));
            }
          }
        }
      } else {
        double g = -INFINITY;
        int pix = INT_MAX, q_best = -1;
        for (int q = lane; q < P; q += 32) {
          const CandRecord* rq = rec_at(a, slot, q);
          double gg = rq->gain;
          int pp = rq->pixel;
          if (pp != INT_MAX && better(gg, pp, g, pix)) { g = gg; pix = pp; q_best = q; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          double og = __shfl_xor_sync(0xffffffffu, g, off);
          int op = __shfl_xor_sync(0xffffffffu, pix, off);
          int oq = __shfl_xor_sync(0xffffffffu, q_best, off);
          if (better(og, op, g, pix)) { g = og; pix = op; q_best = oq; }
        }
        if (q_best >= 0 && g - thr > 0.0) win = q_best;
      }
      if (lane == 0) {
        s_k = win == -2 ? -2 : -1;
        s_pos = 0;
        if (win >= 0) {
          CandRecord rw = *rec_at(a, slot, win);
          s_k = rw.pixel;
          s_pos = (int)rw.key;
          pivot_from_record(rw, a.n_o, s_pv);
          FOR_PORTS(p, a.n_o) s_o[p] = cfma(s_pv.coef, s_pv.Tk[p], s_o[p]);
          s_f = objective_of(s_op, s_o);
        }
      }
      if (a.mode == PNGF_BEST_IMPROVEMENT) {
        __syncwarp();
        const int kb = s_k;
        if (kb >= 0)
          for (int i = lane; i < r; i += 32) {
            c128 al = a.xa[i];
            float2 x = a.X[(size_t)kb * a.R + i];
            float ax = (float)al.x, ay = (float)al.y;
            s_beta[i] = make_float2(fmaf(ax, x.x, -ay * x.y), fmaf(ax, x.y, ay * x.x));
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
    // ---- keep the flip of pixel k
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
      a.xa[r] = s_pv.alpha;
    }
    ++n_acc;
    tick(2);
    mixed_accept_own(a, s_pv, s_beta, r, pb, pe);
    ++r;
    ++since_refresh;
    __syncthreads();
    tick(4);
    if (r == a.R) {
      if (!flush()) { failed = true; break; }
      tick(3);
      if (a.refresh_k > 0 && since_refresh >= a.refresh_k) {
        since_refresh = 0;
        ++n_refresh;
        refresh_x(a, pb, pe);
        if (!grid_sync(ctl)) { failed = true; break; }
        tick(8);
        refresh_residual(a, pb, pe);
        if (!grid_sync(ctl)) { failed = true; break; }
        tick(9);
        refresh_correct(a, pb, pe);
        if (!grid_sync(ctl)) { failed = true; break; }
        tick(10);
        ports_partial(a, pb, pe);
        if (!grid_sync(ctl)) { failed = true; break; }
        tick(11);
        if (threadIdx.x == 0) {
          FOR_PORTS(p, a.n_o) {
            c128 acc = mk(0.0, 0.0);
            for (int q = 0; q < P; ++q) acc = cadd(acc, a.opart[(size_t)q * a.n_o + p]);
            s_o[p] = cadd(a.co[p], acc);
          }
          s_f = objective_of(s_op, s_o);
        }
        __syncthreads();
        tick(5);
      }
    }
    if (status == PNGF_ENUMERIC) break;
    if (a.mode == PNGF_BEST_IMPROVEMENT && n_acc >= max_steps) break;
    if (a.mode == PNGF_FIRST_IMPROVEMENT && t >= n) {
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
  if (a.tensor_fold) {
    if (failed && threadIdx.x < 128) {
      // give what this CTA issued a bounded time to land before the free
      mbar_wait(tcs.mb_load, tcs.ph_load);
      mbar_wait(tcs.mb_mma, tcs.ph_mma);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    tc_free(tcs.tmem);
  }
  if (cta == 0 && threadIdx.x == 0) {
    if (failed) status = PNGF_ETIMEOUT;
    FOR_PORTS(p, a.n_o) ctl->o[p] = s_o[p];
    ctl->f = s_f;
    ctl->since_refresh = since_refresh;
    ctl->r_delay = r;
    ctl->n_acc_total += (int)n_acc;
    ctl->counters[0] = n_acc;
    ctl->counters[1] = n_evals;
    ctl->counters[2] = sweeps_done;
    ctl->counters[3] = converged;
    ctl->counters[4] = n_refresh;
    ctl->counters[5] = n_flush;
    ctl->counters[6] = status;
    ctl->counters[7] = 0;
    ph[7] = clock64() - t_begin;
    for (int q = 0; q < 16; ++q) ctl->phase_cycles[q] = ph[q];
    if (a.counters)
      for (int q = 0; q < 8; ++q) a.counters[q] = ctl->counters[q];
    if (status == PNGF_ENUMERIC || status == PNGF_ETIMEOUT || status == PNGF_EINVAL) latch_status(ctl, status);
  }
}

// ---------------------------------------------------------------- after the factor
__global__ void to_planar_fp32(const c128* __restrict__ W, int n, int ldw, float* __restrict__ Wr,
                               float* __restrict__ Wi, int ldl) {
  int i = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    c128 w = W[(size_t)i * ldw + j];
    Wr[(size_t)i * ldl + j] = (float)w.x;
    Wi[(size_t)i * ldl + j] = (float)w.y;
  }
}

// ---------------------------------------------------------------- single calls
__global__ void mixed_accept_kernel(SweepArgs a, int k) {
  __shared__ Pivot s_pv;
  __shared__ float2 s_beta[kMaxDelay];
  __shared__ int s_r;
  // every CTA rebuilds the pivot from the state of pixel k, which only the
  // owner of k changes, after all CTAs have read it: pixel k's state is read
  // from the snapshot written by accept_snapshot_kernel
  const CandRecord* rk = reinterpret_cast<const CandRecord*>(a.rec);
  if (threadIdx.x == 0) {
    pivot_from_record(*rk, a.n_o, s_pv);
    s_r = a.ctl->r_delay;
  }
  __syncthreads();
  const int r = s_r;
  make_beta(a, k, r, s_beta);
  __syncthreads();
  const int P = gridDim.x, n = a.n;
  const int pb = (int)((long long)n * blockIdx.x / P), pe = (int)((long long)n * (blockIdx.x + 1) / P);
  mixed_accept_own(a, s_pv, s_beta, r, pb, pe);
}

__global__ void accept_snapshot_kernel(SweepArgs a, int k) {
  if (threadIdx.x == 0) {
    CandRecord* rk = reinterpret_cast<CandRecord*>(a.rec);
    fill_record_from_state(a, rk, k);
    Pivot pv;
    pivot_from_record(*rk, a.n_o, pv);
    c128 o[kMaxPorts];
    FOR_PORTS(p, a.n_o) o[p] = cfma(pv.coef, pv.Tk[p], a.ctl->o[p]);
    FOR_PORTS(p, a.n_o) a.ctl->o[p] = o[p];
    a.ctl->f = objective_of(a.op, o);
    a.ctl->n_acc_total += 1;
  }
}

__global__ void accept_finish_kernel(SweepArgs a) {
  if (threadIdx.x == 0) {
    const CandRecord* rk = reinterpret_cast<const CandRecord*>(a.rec);
    Pivot pv;
    pivot_from_record(*rk, a.n_o, pv);
    int r = a.ctl->r_delay;
    a.xa[r] = pv.alpha;
    a.ctl->r_delay = r + 1;
  }
}

__global__ void __launch_bounds__(kThreads) flush_kernel(SweepArgs a) {
  extern __shared__ float dyn_smem[];
  const int r = a.ctl->r_delay;
  if (r < a.R) return;
  flush_tiles(a, r, dyn_smem, blockIdx.x, gridDim.x);
}

__global__ void flush_reset_kernel(SweepArgs a) {
  if (threadIdx.x == 0 && a.ctl->r_delay >= a.R) a.ctl->r_delay = 0;
}


}  // namespace

pngf_status mixed_after_factor(pngf_ctx* c) {
  const int n = c->cfg.n_d;
  dim3 grid((n + 255) / 256 > 8 ? 8 : (n + 255) / 256, n);
  to_planar_fp32<<<grid, 256, 0, c->stream>>>(at<c128>(c, c->L.W), n, c->L.ldw, at<float>(c, c->L.Wlo_re),
                                                at<float>(c, c->L.Wlo_im), c->L.ldl);
  return cuda_status(cudaGetLastError());
}

constexpr size_t kMixedSmem = kFlushSmem > (size_t)TC_SMEM ? kFlushSmem : (size_t)TC_SMEM;

static int mixed_grid(pngf_ctx* c) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(dbs_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMixedSmem);
    cudaFuncSetAttribute(flush_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFlushSmem);
    attr = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dbs_mixed_kernel, kThreads, kMixedSmem);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;
  int g = c->n_sm * per_sm;
  if (c->cfg.n_ctas > 0 && c->cfg.n_ctas < g) g = c->cfg.n_ctas;
  if (g > c->L.n_part) g = c->L.n_part;
  return g;
}

pngf_status run_sweep_mixed(pngf_ctx* c, int n_sweeps, const int32_t* order, int32_t* trace, double* trace_f,
                            int32_t trace_cap, int64_t* counters) {
  SweepArgs a = make_args(c);
  a.n_sweeps = n_sweeps;
  a.order = order;
  a.trace = trace;
  a.trace_f = trace_f;
  a.trace_cap = trace_cap;
  a.counters = counters;
  Control* ctl = a.ctl;
  cudaError_t err = cudaMemsetAsync(&ctl->bar_count, 0, 2 * sizeof(unsigned), c->stream);
  if (err != cudaSuccess) return PNGF_ECUDA;
  err = cudaMemsetAsync(&ctl->sel[0], 0xff, sizeof(ctl->sel), c->stream);
  if (err != cudaSuccess) return PNGF_ECUDA;
  int grid = mixed_grid(c);
  void* params[] = {&a};
  err = cudaLaunchCooperativeKernel((const void*)dbs_mixed_kernel, dim3(grid), dim3(kThreads), params, kMixedSmem,
                                    c->stream);
  return cuda_status(err);
}

pngf_status accept_flip_mixed(pngf_ctx* c, int pixel) {
  SweepArgs a = make_args(c);
  mixed_grid(c);
  accept_snapshot_kernel<<<1, 32, 0, c->stream>>>(a, pixel);
  mixed_accept_kernel<<<c->n_sm, kThreads, 0, c->stream>>>(a, pixel);
  accept_finish_kernel<<<1, 32, 0, c->stream>>>(a);
  if (c->cfg.tensor_fold) {
    pngf_status st = flush_tc_launch(c);
    if (st != PNGF_OK) return st;
  } else {
    flush_kernel<<<c->n_sm, kThreads, kFlushSmem, c->stream>>>(a);
  }
  flush_reset_kernel<<<1, 32, 0, c->stream>>>(a);
  return cuda_status(cudaGetLastError());
}

}  // namespace pngf
