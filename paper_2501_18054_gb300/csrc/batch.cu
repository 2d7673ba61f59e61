// Batched direct binary search: many independent runs in one launch.
//
// The paper notes that independent systems (one per optimisation frequency)
// are updated in parallel with no communication (section "Computational
// efficiency", Table 1 footnote 2); many random starts of DBS on one device
// are independent in the same way.  Here every run is one context (its own
// design region, possibly of a different size, its own W, state and trace),
// and one CTA advances one run at a time through the whole search: scoring,
// selection, the kept-flip update, the FP64 refresh and, on the mixed path,
// the flush of the delayed set, with only CTA-wide barriers.  All runs of a
// batch share one stream.  The runs wait in a queue, largest region first, and
// one CTA per SM takes the next run whenever it finishes one (an atomic
// counter): a large run then has its SM's FP64 pipe to itself, and the small
// runs fill the other SMs (longest-processing-time-first list scheduling).
//
// FIRST mode scores the visiting positions in chunks of blockDim starting at
// the current position and keeps the earliest improving one (the same
// sequential trajectory as scoring all remaining positions, with less
// speculative work when flips are kept often).
#include <cstdio>
#include <memory>
#include <new>
#include <algorithm>
#include <vector>

#include "flush_tc.cuh"
#include "rank1.cuh"

namespace pngf {
namespace {

constexpr int kBatchThreads = 256;

// o = c_o + G_od (v .* e) over all pixels of the run (CTA-local reduction)
__device__ void cta_ports(const SweepArgs& a, const ObjParams& op, c128* s_o, double* s_f) {
  __shared__ c128 red[kBatchThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int p = 0; p < a.n_o; ++p) {
    c128 acc = mk(0.0, 0.0);
    for (int j = threadIdx.x; j < a.n; j += blockDim.x)
      acc = cfma(a.God[(size_t)p * a.n + j], cmul(a.v[j], a.e[j]), acc);
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
    }
    __syncthreads();
    if (lane == 0) red[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      c128 sum = mk(0.0, 0.0);
      for (int q = 0; q < nw; ++q) sum = cadd(sum, red[q]);
      s_o[p] = cadd(a.co[p], sum);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *s_f = objective_of(op, s_o);
  __syncthreads();
}

__device__ void cta_refresh(const SweepArgs& a, const ObjParams& op, c128* s_o, double* s_f) {
  __syncthreads();
  refresh_x(a, 0, a.n);
  __syncthreads();
  refresh_residual(a, 0, a.n);
  __syncthreads();
  refresh_correct(a, 0, a.n);
  __syncthreads();
  cta_ports(a, op, s_o, s_f);
}

__global__ void __launch_bounds__(kBatchThreads, 2) dbs_batch_kernel(const SweepArgs* __restrict__ runs, int n_runs,
                                                                      int* __restrict__ queue) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ c128 s_o[kMaxPorts];
  __shared__ double s_f;
  __shared__ ObjParams s_op;
  __shared__ Pivot s_pv;
  __shared__ float2 s_beta[kMaxDelay];
  __shared__ int s_k;
  __shared__ long long s_best;
  // tensor-core fold (tiles of 128 x 64): this CTA holds tc_tmem_cols(1) columns of tensor memory for all its runs
  __shared__ __align__(8) unsigned long long s_tc_bars[TC_NBAR];
  __shared__ unsigned s_tmem;
  const bool use_tc = n_runs > 0 && runs[0].tensor_fold;
  TcState tcs{};
  if (use_tc) tc_setup(tcs, s_tc_bars, &s_tmem, tc_tmem_cols(1));
  bool tc_failed = false;
  __shared__ int s_run;
  while (!tc_failed) {
    __syncthreads();  // every thread has read the previous s_run
    if (threadIdx.x == 0) s_run = atomicAdd(queue, 1);
    __syncthreads();
    const int run = s_run;
    if (run >= n_runs) break;
    const SweepArgs& a = runs[run];
    const int n = a.n;
    Control* ctl = a.ctl;
    __syncthreads();
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
    int s = 0, t = 0, acc_in_sweep = 0;
    const long long E = (long long)n * (n + 1) / 2;
    c128* cs = reinterpret_cast<c128*>(dyn);  // FP64 path: the gathered column c, then alpha c
    c128* acs = cs + n;
    while (true) {
      const double f = s_f;
      const double thr = accept_threshold(s_op, f);
      // ---- score a chunk of positions (FIRST) or every pixel (BEST)
      long long best = LLONG_MAX;
      double g = -INFINITY;
      int pix = INT_MAX;
      c128 b_alpha = mk(0.0, 0.0), b_coef = b_alpha;
      if (a.mode == PNGF_FIRST_IMPROVEMENT) {
        const int q = t + threadIdx.x;
        if (q < n) {
          const int j = a.order ? a.order[(size_t)s * n + q] : q;
          double fn;
          c128 al, co;
          if ((unsigned)j < (unsigned)n && score_pixel(a, s_op, j, s_o, fn, nullptr, &al, &co) &&
              gain_of(s_op, fn, f) - thr > 0.0) {
            best = q;
            pix = j;
            b_alpha = al;
            b_coef = co;
          }
          if ((unsigned)j >= (unsigned)n) status = PNGF_EINVAL;
        }
        long long bmin = block_min_ll(best);
        if (bmin != LLONG_MAX && best == bmin) {
          s_k = pix;
          s_best = bmin;
          s_pv.k = pix;
          s_pv.alpha = b_alpha;
          s_pv.coef = b_coef;
          for (int p = 0; p < a.n_o; ++p) s_pv.Tk[p] = a.T[(size_t)p * a.ldt + pix];
        }
        if (threadIdx.x == 0 && bmin == LLONG_MAX) s_k = -1;
        __syncthreads();
        if (__syncthreads_or(status == PNGF_EINVAL)) {
          status = PNGF_EINVAL;
          break;
        }
        if (s_k < 0) {
          const int chunk_end = min(n, t + (int)blockDim.x);
          n_evals += chunk_end - t;
          t = chunk_end;
          if (t < n) continue;
          ++sweeps_done;
          if (acc_in_sweep == 0) { converged = 1; break; }
          ++s;
          if (s >= a.n_sweeps) break;
          t = 0;
          acc_in_sweep = 0;
          continue;
        }
        const int q_star = (int)s_best;
        n_evals += q_star - t + 1;
        t = q_star + 1;
      } else {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          double fn;
          c128 al, co;
          if (!score_pixel(a, s_op, j, s_o, fn, nullptr, &al, &co)) continue;
          double gg = gain_of(s_op, fn, f);
          if (better(gg, j, g, pix)) { g = gg; pix = j; b_alpha = al; b_coef = co; }
        }
        double gb = g;
        int pb2 = pix;
        block_best(gb, pb2);
        if (pb2 != INT_MAX && gb - thr > 0.0 && pix == pb2) {
          s_k = pix;
          s_pv.k = pix;
          s_pv.alpha = b_alpha;
          s_pv.coef = b_coef;
          for (int p = 0; p < a.n_o; ++p) s_pv.Tk[p] = a.T[(size_t)p * a.ldt + pix];
        }
        if (threadIdx.x == 0 && !(pb2 != INT_MAX && gb - thr > 0.0)) s_k = -1;
        __syncthreads();
        n_evals += n;
        ++sweeps_done;
        if (s_k < 0) { converged = 1; break; }
      }
      // ---- keep the flip of pixel k
      const int k = s_k;
      if (threadIdx.x == 0) {
        FOR_PORTS(p, a.n_o) s_o[p] = cfma(s_pv.coef, s_pv.Tk[p], s_o[p]);
        s_f = objective_of(s_op, s_o);
        if (n_acc < a.trace_cap) {
          if (a.trace) {
            int32_t* tr = a.trace + 4 * n_acc;
            tr[0] = a.mode == PNGF_FIRST_IMPROVEMENT ? s : (int)n_acc;
            tr[1] = a.mode == PNGF_FIRST_IMPROVEMENT ? t - 1 : 0;
            tr[2] = k;
            tr[3] = 0;
          }
          if (a.trace_f) a.trace_f[n_acc] = s_f;
        } else if (status == PNGF_OK) {
          status = PNGF_ECAPACITY;
        }
        if (a.mixed) a.xa[r] = s_pv.alpha;
      }
      ++n_acc;
      ++acc_in_sweep;
      if (!a.mixed) {
        // FP64: gather c = W[:,k] into shared memory, then the state and rank-1 updates
        for (int j = threadIdx.x; j < n; j += blockDim.x)
          cs[j] = (j >= k) ? a.W[(size_t)k * a.ldw + j] : a.W[(size_t)j * a.ldw + k];
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          c128 cj = cs[j];
          c128 aj = cmul(s_pv.alpha, cj);
          acs[j] = aj;
          a.diag[j] = cfma(aj, cj, a.diag[j]);
          a.e[j] = cfma(s_pv.coef, cj, a.e[j]);
          for (int p = 0; p < a.n_o; ++p) {
            c128* tp = a.T + (size_t)p * a.ldt + j;
            *tp = cfma(aj, s_pv.Tk[p], *tp);
          }
          if (j == k) {
            uint8_t nb = a.b[j] ^ 1;
            a.b[j] = nb;
            a.v[j] = nb ? a.dv[j] : mk(0.0, 0.0);
          }
        }
        __syncthreads();  // every alpha c_j formed
        rank1_upper_ac(a.W, n, a.ldw, acs, cs, 0, E);
        __syncthreads();
        ++since_refresh;
        if (a.refresh_k > 0 && since_refresh >= a.refresh_k) {
          since_refresh = 0;
          ++n_refresh;
          cta_refresh(a, s_op, s_o, &s_f);
        }
      } else {
        // mixed: beta, column assembly from the FP32 copy, FP64 state update
        for (int i = threadIdx.x; i < r; i += blockDim.x) {
          c128 al = a.xa[i];
          float2 x = a.X[(size_t)k * a.R + i];
          float ax = (float)al.x, ay = (float)al.y;
          s_beta[i] = make_float2(fmaf(ax, x.x, -ay * x.y), fmaf(ax, x.y, ay * x.x));
        }
        __syncthreads();
        mixed_accept_own(a, s_pv, s_beta, r, 0, n);
        ++r;
        ++since_refresh;
        if (r == a.R) {
          __syncthreads();
          if (use_tc) {
            tc_prepare(a, r, a.tcimgA, a.tcimgB, threadIdx.x, blockDim.x);
            __threadfence_block();
            __syncthreads();
            if (!tc_fold_tiles<1>(a, r, a.tcimgA, a.tcimgB, dyn, tcs, 0, 1)) {
              status = PNGF_ETIMEOUT;
              tc_failed = true;
              break;
            }
          } else {
            flush_tiles(a, r, reinterpret_cast<float*>(dyn), 0, 1);
          }
          __syncthreads();
          r = 0;
          ++n_flush;
          if (a.refresh_k > 0 && since_refresh >= a.refresh_k) {
            since_refresh = 0;
            ++n_refresh;
            cta_refresh(a, s_op, s_o, &s_f);
          }
        }
      }
      if (!isfinite(s_f)) {
        status = PNGF_ENUMERIC;
        break;
      }
      if (a.mode == PNGF_BEST_IMPROVEMENT && n_acc >= a.n_sweeps) break;
      if (a.mode == PNGF_FIRST_IMPROVEMENT && t >= n) {
        ++sweeps_done;
        ++s;
        if (s >= a.n_sweeps) break;
        t = 0;
        acc_in_sweep = 0;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      FOR_PORTS(p, a.n_o) ctl->o[p] = s_o[p];
      ctl->f = s_f;
      ctl->since_refresh = since_refresh;
      ctl->r_delay = r;
      ctl->n_acc_total += (int)n_acc;
      long long cnt[8] = {n_acc, n_evals, sweeps_done, converged, n_refresh, n_flush, status, 0};
      for (int q = 0; q < 8; ++q) ctl->counters[q] = cnt[q];
      if (a.counters)
        for (int q = 0; q < 8; ++q) a.counters[q] = cnt[q];
      if (status == PNGF_ENUMERIC || status == PNGF_EINVAL || status == PNGF_ETIMEOUT) latch_status(ctl, status);
    }
  }
  if (use_tc) tc_teardown(tcs, tc_failed);
}

// The per-run argument table is written by the device from kernel parameters
// (chunks of the table passed by value), so that no host buffer has to outlive
// the call: a stream capture records the values themselves.
constexpr int kArgChunk = 30000 / (int)sizeof(SweepArgs);
struct ArgChunk {
  SweepArgs a[kArgChunk];
  int count;
};
static_assert(kArgChunk >= 1 && sizeof(ArgChunk) <= 32000, "kernel parameter space");

__global__ void write_args_kernel(const ArgChunk ch, SweepArgs* __restrict__ dst) {
  for (int i = threadIdx.x; i < ch.count; i += blockDim.x) dst[i] = ch.a[i];
}

}  // namespace

// the argument table, then the run queue's counter
static size_t batch_table_bytes(int n_runs) { return ((size_t)n_runs * sizeof(SweepArgs) + 255) / 256 * 256; }
size_t batch_workspace_bytes(int n_runs) { return batch_table_bytes(n_runs) + 256; }

pngf_status run_sweep_batch(pngf_ctx* const* ctxs, int n_runs, int n_sweeps, const int32_t* const* orders,
                            int32_t* const* traces, double* const* trace_f, int32_t trace_cap, int64_t* counters,
                            void* ws, size_t ws_bytes) {
  pngf_ctx* c0 = ctxs[0];
  SweepArgs* table = static_cast<SweepArgs*>(ws);
  int* queue = reinterpret_cast<int*>(static_cast<unsigned char*>(ws) + batch_table_bytes(n_runs));
  std::unique_ptr<ArgChunk> ch(new (std::nothrow) ArgChunk());
  if (!ch) return PNGF_ENOMEM;
  // queue order: largest region first (ties: the caller's order)
  std::vector<int> rank(n_runs);
  for (int r = 0; r < n_runs; ++r) rank[r] = r;
  std::stable_sort(rank.begin(), rank.end(), [&](int x, int y) { return ctxs[x]->cfg.n_d > ctxs[y]->cfg.n_d; });
  int max_n = 0;
  for (int r0 = 0; r0 < n_runs; r0 += kArgChunk) {
    ch->count = n_runs - r0 < kArgChunk ? n_runs - r0 : kArgChunk;
    for (int i = 0; i < ch->count; ++i) {
      const int r = rank[r0 + i];
      SweepArgs a = make_args(ctxs[r]);
      a.n_sweeps = n_sweeps;
      a.order = orders ? orders[r] : nullptr;
      a.trace = traces ? traces[r] : nullptr;
      a.trace_f = trace_f ? trace_f[r] : nullptr;
      a.trace_cap = trace_cap;
      a.counters = counters ? counters + 8 * (size_t)r : nullptr;
      ch->a[i] = a;
      if (a.n > max_n) max_n = a.n;
    }
    write_args_kernel<<<1, 128, 0, c0->stream>>>(*ch, table + r0);
    if (cudaGetLastError() != cudaSuccess) return PNGF_ECUDA;
  }
  const bool mixed = c0->cfg.precision == PNGF_MIXED;
  size_t smem = mixed ? (kFlushSmem > (size_t)tc_fold_smem(1) ? kFlushSmem : (size_t)tc_fold_smem(1))
                      : 2 * (size_t)max_n * sizeof(c128);
  if (cudaFuncSetAttribute(dbs_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PNGF_ECUDA;
  if (cudaMemsetAsync(queue, 0, sizeof(int), c0->stream) != cudaSuccess) return PNGF_ECUDA;
  int grid = c0->n_sm;  // one CTA per SM
  if (grid > n_runs) grid = n_runs;
  dbs_batch_kernel<<<grid, kBatchThreads, smem, c0->stream>>>(static_cast<const SweepArgs*>(ws), n_runs, queue);
  return cuda_status(cudaGetLastError());
}

}  // namespace pngf
