// Direct binary search on the device, mixed-precision path.
//
// The maintained inverse W = M^-1 G (the paper's C~^-1, Supplementary Note 4)
// is kept as a planar FP32 copy W_lo plus a delayed rank-r correction:
//   W = W_lo + sum_{i<r} alpha_i x_i x_i^T,   x_i = column of W at kept flip i.
// Per kept flip of pixel k only the column c = W[:,k] is needed:
//   c_j = W_lo(k, j) + sum_{i<r} (alpha_i x_i[k]) x_i[j]      (FP32 arithmetic)
// which updates diag(W), e and T and is appended to the delayed set.  What
// decides a flip, diag(W), e, T, o, the Sherman-Morrison denominators d_k and
// alpha (Eqs. 9 and 14), is carried as double-words (FP32 pairs, ~48 bits,
// dd.cuh), so the whole per-flip chain runs on the FP32 pipe: on GB300 the
// FP64 pipe retires one warp instruction per 64 cycles on each SM
// sub-partition.  Every R kept flips the delayed set is folded into W_lo with
// one rank-R product over the upper triangle on the tensor cores (the paper's
// O(N_opt^2) update of Supplementary Note 3, done once per R flips), and every
// refresh_k flips e and T are refined against G with a double-float residual.
//
// Each CTA publishes its best candidate together with the pixel state the
// pivot needs, and the CTAs agree on the kept flip by exchanging one word
// each: no grid barrier per kept flip, only around the fold and the refresh.
#include <cstdio>

#include "flush_tc.cuh"
#include "refresh_df.cuh"
#include "dd.cuh"

namespace pngf {
namespace {

// ---------------------------------------------------------------- persistent mixed DBS
// Per kept flip the CTAs exchange one 64-bit word each instead of meeting at a
// grid barrier: word = round sequence number << 44 | candidate key, with key =
// position << 22 | pixel (FIRST mode) or pixel (BEST mode, gain in the
// record); every CTA waits for all P words of the round, reduces them itself
// and fetches the winner's record, the winner's delayed row X[k] and
// W_lo(k, own) in one parallel round trip.  Words and records alternate
// between two buffers by round parity: a CTA can run at most one round ahead
// of the slowest reader, so the buffer it writes is never one still being read.
//
// The state of a CTA's own pixels (diag W, e, T, b, visiting position and the
// delayed rows X[own]) lives in shared memory between refreshes; only b and v
// of the flipped pixel and the appended column of X are written through.
//
// The per-flip chain is kept short: the score needs one reciprocal,
//   alpha_j = 1 / z_j,  z_j = 1/delta_j - W_jj   (= delta_j / d_j, Eq. 14),
// with 1/delta_j = -+1/dv_j tabulated, the rows of T are kept pre-multiplied by
// the port scales so that S_p(new) = S_p + coef T'_p,j is one complex FMA,
// the winner's record carries f(new) (every CTA forms S(new) with the same
// operations the scorer used, off the critical path), and the state update
// spreads diag, e and the rows of T over warps of different sub-partitions.
// FP64 appears only at set-up, after a refresh, before a fold (alpha for the
// fold's operands) and at the end (state, trace objectives).
constexpr int kOwnMax = 256;                                       // pixels per CTA, at most
constexpr int kSlotStride = 16;                                    // 64-bit words between two CTAs' words
constexpr int kSeqShift = 44;
constexpr int kPixBits = 22;
constexpr unsigned long long kKeyMask = (1ull << kSeqShift) - 1;
constexpr long long kNoCand = (long long)kKeyMask;                 // above every real key
constexpr unsigned kSeqMask = (1u << (64 - kSeqShift)) - 1;
constexpr int kPartsMax = 8;                                       // warps per 32 pixels in the delayed sum
// Own state at the start of the dynamic shared memory, one row of `oss` entries
// each (oss = the launch's largest own-pixel count rounded up to 32): T'[n_o],
// diag, e, dv, 1/dv (16 B), |dv|^2 (8 B); sized per launch, 1024-B aligned so
// that the fold's operand buffers after it stay aligned.
__host__ __device__ constexpr size_t own_state_bytes(int n_o, int oss) {
  return (((size_t)(n_o + 4) * oss * sizeof(c128) + (size_t)oss * sizeof(double)) + 1023) / 1024 * 1024;
}
__host__ __device__ constexpr int own_stride(int n, int grid) { return ((n + grid - 1) / grid + 31) & ~31; }
constexpr size_t cmax(size_t x, size_t y) { return x > y ? x : y; }
// the work area: the fold's operand buffers and stage (during a fold); the
// delayed rows of the own pixels (R x oss float2) and the delayed sum's partials
// (kPartsMax x oss float2) between folds; the refresh's list, ring and staging
constexpr size_t kMixedWork = cmax(kFlushSmem, (size_t)tc_fold_smem(2));
__host__ __device__ constexpr size_t delayed_rows_bytes(int R, int oss) {
  return ((size_t)R + kPartsMax) * oss * sizeof(float2);
}
static_assert(kMixedWork >= (size_t)32768 * sizeof(int), "active-pixel list of the refresh (n_d <= 32768)");
static_assert(kMixedWork >= cs_min_smem_bytes(1 + kMaxPorts), "staging of the refresh correction");
// dynamic + static (~17 KB) shared memory: with the own state of 108 pixels
// (4 runs of 4096) or 216 (8 runs) and two ports, within the 196 KB carve-out,
// which leaves 60 KB of L1 for the kernel's local-memory spills and global reads
// a refresh holds the active list (n ints) and then the residual's copy ring
// (its partial sums, kThreads float4, reuse the ring) in the work area
__host__ __device__ constexpr size_t rd_list_bytes(int n) { return ((size_t)n * 4 + 15) / 16 * 16; }

// a CTA's candidate of one round, with everything the other CTAs need to keep it
struct MixRecord {
  long long key;  // FIRST: visiting position
  double gain;    // BEST: gain of the candidate
  dd f_new;       // objective after the flip
  int pixel;
  int b;
  cdd alpha, coef;
  cdd Tk[kMaxPorts];  // scaled rows T'_p at the pixel
};
static_assert(sizeof(MixRecord) <= kRecordBytes, "record slot");
static_assert(offsetof(MixRecord, f_new) % 8 == 0 && offsetof(MixRecord, alpha) % 8 == 0 &&
                  offsetof(MixRecord, coef) % 8 == 0 && offsetof(MixRecord, Tk) % 8 == 0,
              "record words: every double-word on its own 8-byte word");

// the pivot of a kept flip, as every CTA holds it
struct MixPivot {
  int k;
  cdd alpha, coef;  // coef = alpha e_k
  cdd Tk[kMaxPorts];
};

// FP64 <-> double-word conversions (FP64 instructions: used at set-up, after a
// refresh and at the end, never on the per-flip chain)
__device__ __forceinline__ dd dd_from(double x) {
  const float hi = (float)x;
  return dd{hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ cdd cdd_from(c128 x) { return cdd{dd_from(x.x), dd_from(x.y)}; }
__device__ __forceinline__ double dd_to(dd x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ c128 cdd_to(cdd x) { return mk(dd_to(x.re), dd_to(x.im)); }

__device__ __forceinline__ MixRecord* mrec_at(const SweepArgs& a, int par, int q) {
  return reinterpret_cast<MixRecord*>(a.rec) + (size_t)par * gridDim.x + q;
}

__device__ __forceinline__ int owner_of(int k, int n, int P) { return (int)(((long long)(k + 1) * P - 1) / n); }

// acc + the objective term of one port from |S_p|^2 (w_p |S_p|^2, or
// w_p (1 - |S_p|)^2), in double-words; the objective kind is a template
// parameter so that the other kind's instructions are not issued per pixel
template <int OBJ>
__device__ __forceinline__ dd obj_acc(dd w, dd a2, dd acc) {
  if (OBJ == PNGF_OBJ_MAX_WEIGHTED_POWER) return dd_add(acc, dd_mul(w, a2));
  const dd m = dd_sub(dd_of(1.0f), dd_sqrt(a2));
  return dd_add(acc, dd_mul(w, dd_mul(m, m)));
}
// improvement bound f + thr (maximised) or f - thr (minimised), thr = tau max(|f|, 1e-30)
template <int OBJ>
__device__ __forceinline__ dd improve_bound(dd f, dd tau) {
  const dd af = dd_abs(f);
  const dd thr = dd_mul(af.hi > 1e-30f ? af : dd_of(1e-30f), tau);
  return OBJ == PNGF_OBJ_MAX_WEIGHTED_POWER ? dd_add(f, thr) : dd_sub(f, thr);
}

// waits (bounded) for CTA q's word of round `seq`; returns its key
__device__ __forceinline__ long long poll_word(const unsigned long long* w, unsigned seq, bool& ok,
                                               unsigned long long lim) {
  unsigned long long it = 0;
  const unsigned long long t0 = global_ns();
  for (;;) {
    unsigned long long v = *reinterpret_cast<const volatile unsigned long long*>(w);
    if ((unsigned)(v >> kSeqShift) == seq) return (long long)(v & kKeyMask);
    if (++it > lim || ((it & 63) == 0 && global_ns() - t0 > kWaitNs)) {
      ok = false;
      return kNoCand;
    }
    if (it > 1024) __nanosleep(32);  // the awaited word usually lands within a few round trips
  }
}

template <int OBJ>
__global__ void __launch_bounds__(kThreads) dbs_mixed_kernel(SweepArgs a) {
  extern __shared__ float dyn_smem[];
  const int P = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int n = a.n, n_o = a.n_o;
  const int pb = (int)((long long)n * cta / P), pe = (int)((long long)n * (cta + 1) / P);
  const int own = pe - pb;
  Control* ctl = a.ctl;
  const unsigned long long spin_lim = spin_limit_of(ctl);
  hold_if_asked(ctl);
  // own-pixel state (thread jl < own scores pixel pb + jl)
  // (double-words, so that the per-flip chain runs on the FP32 pipe; dv itself stays FP64)
  const int OSS = own_stride(n, P);  // row stride of the own state (the same in every CTA)
  const size_t state_bytes = own_state_bytes(n_o, OSS);
  cdd* s_T = reinterpret_cast<cdd*>(dyn_smem);  // [n_o][OSS], T'_p,j = T_p,j scale_p
  cdd* s_diag = s_T + n_o * OSS;
  cdd* s_e = s_diag + OSS;
  c128* s_dv = reinterpret_cast<c128*>(s_e + OSS);
  cdd* s_idv = reinterpret_cast<cdd*>(s_dv + OSS);             // 1 / dv (0 where dv = 0)
  dd* s_dv2 = reinterpret_cast<dd*>(s_idv + OSS);                // |dv|^2
  unsigned char* work = reinterpret_cast<unsigned char*>(dyn_smem) + state_bytes;
  __shared__ int s_pos[kOwnMax];
  __shared__ unsigned char s_b[kOwnMax];
  __shared__ float2 s_wk[kOwnMax];
  __shared__ float2 s_c[kOwnMax];  // column entry c_j of the kept flip (FP32)
  __shared__ cdd s_ac[kOwnMax];     // alpha c_j
  __shared__ float2 s_beta[kMaxDelay], s_alpha[kMaxDelay];
  __shared__ cdd s_S[kMaxPorts];       // scaled port amplitudes S_p = (o_p - off_p) scale_p
  __shared__ dd s_w[kMaxPorts], s_tau;  // objective weights w_p, acceptance tolerance tau
  __shared__ c128 s_o[kMaxPorts];      // port amplitudes after a refresh
  __shared__ c128 s_iscale[kMaxPorts];  // 1 / scale_p
  __shared__ dd s_f, s_fthr;  // objective, improvement bound
  __shared__ MixPivot s_pv;
  __shared__ ObjParams s_op;
  __shared__ int s_fail, s_bad;
  // delayed columns of the own pixels between folds, column-major: Xs[i * OS + jl] = x_i[pb + jl]
  float2* Xs = reinterpret_cast<float2*>(work);
  // partial delayed sums of the update (U2), after the largest Xs; dead during a fold
  const int OS = (own + 31) & ~31;
  const int R = a.R;
  float2* s_part = reinterpret_cast<float2*>(work + (size_t)R * OSS * sizeof(float2));
  int r = ctl->r_delay;
  if (tid == 0) {
    s_op = a.op;
    FOR_PORTS(p, n_o) {
      s_iscale[p] = cdiv(mk(1.0, 0.0), a.op.scale[p]);
      s_S[p] = cdd_from(cmul(csub(ctl->o[p], a.op.off[p]), a.op.scale[p]));
      s_w[p] = dd_from(a.op.w[p]);
    }
    s_tau = dd_from(a.op.tau);
    s_f = dd_from(ctl->f);
    const double thr = accept_threshold(a.op, ctl->f);
    s_fthr = dd_from(OBJ == PNGF_OBJ_MAX_WEIGHTED_POWER ? ctl->f + thr : ctl->f - thr);
    s_fail = 0;
  }
  for (int jl = tid; jl < own; jl += blockDim.x) {
    const int j = pb + jl;
    const c128 dv = a.dv[j];
    s_diag[jl] = cdd_from(a.diag[j]);
    s_e[jl] = cdd_from(a.e[j]);
    s_dv[jl] = dv;
    s_dv2[jl] = dd_from(cabs2(dv));
    s_idv[jl] = cdd_from(cabs2(dv) > 0.0 ? cdiv(mk(1.0, 0.0), dv) : mk(0.0, 0.0));
    s_b[jl] = a.b[j];
    for (int p = 0; p < n_o; ++p)
      s_T[p * OSS + jl] = cdd_from(cmul(a.T[(size_t)p * a.ldt + j], a.op.scale[p]));
    if (!a.order) s_pos[jl] = j;
  }
  for (int q = tid; q < own * r; q += blockDim.x) {
    const int jl = q / r, i = q - jl * r;
    Xs[i * OS + jl] = a.X[(size_t)(pb + jl) * R + i];
  }
  for (int i = tid; i < r; i += blockDim.x) {
    c128 al = a.xa[i];
    s_alpha[i] = make_float2((float)al.x, (float)al.y);
  }
  __syncthreads();
  auto store_et = [&](bool with_diag) {
    for (int jl = tid; jl < own; jl += blockDim.x) {
      const int j = pb + jl;
      a.e[j] = cdd_to(s_e[jl]);
      if (with_diag) a.diag[j] = cdd_to(s_diag[jl]);
      for (int p = 0; p < n_o; ++p) a.T[(size_t)p * a.ldt + j] = cmul(cdd_to(s_T[p * OSS + jl]), s_iscale[p]);
    }
  };
  auto load_et = [&]() {
    for (int jl = tid; jl < own; jl += blockDim.x) {
      const int j = pb + jl;
      s_e[jl] = cdd_from(a.e[j]);
      for (int p = 0; p < n_o; ++p) s_T[p * OSS + jl] = cdd_from(cmul(a.T[(size_t)p * a.ldt + j], s_op.scale[p]));
    }
  };
  auto load_pos = [&]() {
    for (int jl = tid; jl < own; jl += blockDim.x) s_pos[jl] = a.pos_of[pb + jl];
  };
  long long n_acc = 0, n_evals = 0, n_refresh = 0, n_flush = 0, sum_active = 0;
  int sweeps_done = 0, converged = 0, status = PNGF_OK;
  int since_refresh = ctl->since_refresh;
  int s = 0, t = 0, acc_in_sweep = 0;
  long long round = 0;
  bool failed = false;
  const bool timer = (cta == 0 && tid == 0);
  __shared__ long long ph[16];  // phase cycles, kept by the timer thread only
  if (timer)
    for (int q = 0; q < 16; ++q) ph[q] = 0;
  long long t_last = clock64(), t_begin = t_last;
  auto tick = [&](int phase) {
    if (timer) {
      long long now = clock64();
      ph[phase] += now - t_last;
      t_last = now;
    }
  };
  // writes the positions of sweep sw for the visiting positions [pb, pe);
  // every CTA then reads its own pixels' positions after a barrier
  auto setup_sweep = [&](int sw) -> bool {
    for (int q = pb + tid; q < pe; q += blockDim.x) {
      int px = a.order[(size_t)sw * n + q];
      if ((unsigned)px < (unsigned)n) a.pos_of[px] = q;
      else latch_status(ctl, PNGF_EINVAL);
    }
    if (!grid_sync(ctl)) return false;
    if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) status = PNGF_EINVAL;
    load_pos();
    return true;
  };
  // tensor-core fold (tiles of 128 x 128): warp 0 holds all 512 columns of tensor memory for the whole search
  __shared__ __align__(8) unsigned long long s_tc_bars[TC_NBAR];
  __shared__ unsigned s_tmem;
  TcState tcs{};
  if (a.tensor_fold) tc_setup(tcs, s_tc_bars, &s_tmem, tc_tmem_cols(2));
  // the fold reuses the shared memory of the delayed rows: they are in global
  // X as well and the delayed set is empty afterwards
  // alpha_i kept since the last fold (or this call's start) as double-words -> FP64 xa
  int r_dd = r;  // first entry of xadd written by this call
  auto alpha_to_fp64 = [&]() {
    if (cta == 0)
      for (int i = r_dd + tid; i < r; i += blockDim.x) a.xa[i] = cdd_to(reinterpret_cast<const cdd*>(a.xadd)[i]);
    r_dd = 0;
  };
  auto flush = [&]() -> bool {
    alpha_to_fp64();  // before the barrier that publishes it to every CTA's fold
    if (!grid_sync(ctl)) return false;
    if (a.tensor_fold) {
      tc_prepare(a, r, a.tcimgA, a.tcimgB, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                 (long long)gridDim.x * blockDim.x);
      if (!grid_sync(ctl)) return false;
      tick(14);
      if (!tc_fold_tiles<2>(a, r, a.tcimgA, a.tcimgB, work, tcs, blockIdx.x, gridDim.x)) {
        if (threadIdx.x == 0) latch_status(ctl, PNGF_ETIMEOUT);
        return false;
      }
    } else {
      flush_tiles(a, r, reinterpret_cast<float*>(work), blockIdx.x, gridDim.x);
    }
    if (!grid_sync(ctl)) return false;
    r = 0;
    ++n_flush;
    return true;
  };
  if (a.mode == PNGF_FIRST_IMPROVEMENT && a.order) {
    if (!setup_sweep(0)) failed = true;
    __syncthreads();
  }
  const long long max_steps = a.n_sweeps;
  while (!failed && status != PNGF_EINVAL) {
    // improving: f_new > f + thr (maximised) or f_new < f - thr (minimised); the
    // bound is formed once per kept flip by the thread that sets f
    const dd fthr = s_fthr;
    const int par = (int)(round & 1);
    const unsigned seq = (unsigned)((round + 1) & kSeqMask);
    unsigned long long* words = a.slots + (size_t)par * P * kSlotStride;
    // ---- score own pixels; the CTA's best candidate goes to its record, its key to its word
    long long key = kNoCand;
    {
      dd fn = dd_of(0.0f);
      cdd al = cdd_of(0.0f, 0.0f), co = al;
      bool ok = false;
      if (tid < own) {  // in double-words on the FP32 pipe
        const cdd idv = s_idv[tid], w = s_diag[tid];
        const cdd z = s_b[tid] ? cdd_sub(cdd{dd_neg(idv.re), dd_neg(idv.im)}, w) : cdd_sub(idv, w);
        const dd z2 = cdd_abs2(z);
        if (!(z2.hi * s_dv2[tid].hi < 1e-28f)) {  // |d_j| = |delta_j| |z_j|; singular candidates are skipped
          const dd iz = dd_rcp(z2);
          al = cdd{dd_mul(z.re, iz), dd_neg(dd_mul(z.im, iz))};
          co = cdd_mul(al, s_e[tid]);
          // ports two at a time: their |S_p(new)|^2 chains are independent, the
          // objective still adds them in port order
          int p = 0;
#pragma unroll 1
          for (; p + 1 < n_o; p += 2) {
            const dd a0 = cdd_abs2(cdd_fma(co, s_T[p * OSS + tid], s_S[p]));
            const dd a1 = cdd_abs2(cdd_fma(co, s_T[(p + 1) * OSS + tid], s_S[p + 1]));
            fn = obj_acc<OBJ>(s_w[p + 1], a1, obj_acc<OBJ>(s_w[p], a0, fn));
          }
          if (p < n_o) fn = obj_acc<OBJ>(s_w[p], cdd_abs2(cdd_fma(co, s_T[p * OSS + tid], s_S[p])), fn);
          ok = true;
        }
      }
      MixRecord* rc = mrec_at(a, par, cta);
      auto fill = [&](long long kk, double gg) {
        rc->key = kk;
        rc->gain = gg;
        rc->f_new = fn;
        rc->pixel = pb + tid;
        rc->b = s_b[tid];
        rc->alpha = al;
        rc->coef = co;
        for (int p = 0; p < n_o; ++p) rc->Tk[p] = s_T[p * OSS + tid];
      };
      if (a.mode == PNGF_FIRST_IMPROVEMENT) {
        long long cand = kNoCand;
        if (ok) {
          const int pos = s_pos[tid];
          const bool improving = OBJ == PNGF_OBJ_MAX_WEIGHTED_POWER ? dd_gt(fn, fthr) : dd_lt(fn, fthr);
          if (pos >= t && improving) cand = ((long long)pos << kPixBits) | (pb + tid);
        }
        key = block_min_ll(cand);
        if (key != kNoCand && cand == key) fill(cand >> kPixBits, 0.0);
      } else {
        double g = -INFINITY;
        int pix = INT_MAX;
        if (ok) {
          const dd f = s_f;
          g = dd_to(OBJ == PNGF_OBJ_MAX_WEIGHTED_POWER ? dd_sub(fn, f) : dd_sub(f, fn));
          pix = pb + tid;
        }
        double gb = g;
        int pb2 = pix;
        block_best(gb, pb2);
        if (pb2 != INT_MAX) {
          key = pb2;
          if (pix == pb2) fill(0, gb);
        }
      }
    }
    tick(0);
    __syncthreads();
    if (tid == 0) {
      fence_acq_rel_gpu();  // release: the record and the earlier appends to X before the word
      *reinterpret_cast<volatile unsigned long long*>(words + (size_t)cta * kSlotStride) =
          ((unsigned long long)seq << kSeqShift) | (unsigned long long)key;
    }
    tick(12);
    // ---- every CTA's word of this round
    int k = -1, pos_k = 0;
    {
      long long kq = kNoCand;
      if (tid < P) {
        bool ok = true;
        kq = poll_word(words + (size_t)tid * kSlotStride, seq, ok, spin_lim);
        if (!ok) {
          s_fail = 1;
          latch_status(ctl, PNGF_ETIMEOUT);
        }
        fence_acq_rel_gpu();  // acquire: CTA q's record and appends to X
      }
      if (a.mode == PNGF_FIRST_IMPROVEMENT) {
        const long long kmin = block_min_ll(kq);
        if (kmin != kNoCand) {
          pos_k = (int)(kmin >> kPixBits);
          k = (int)(kmin & ((1 << kPixBits) - 1));
        }
      } else {
        double g = -INFINITY;
        int pix = INT_MAX;
        if (kq != kNoCand) {
          pix = (int)kq;
          g = mrec_at(a, par, tid)->gain;
        }
        block_best(g, pix);
        // the best candidate is kept when it clears the improvement bound
        if (pix != INT_MAX) {
          const dd fb = mrec_at(a, par, owner_of(pix, n, P))->f_new;
          if (OBJ == PNGF_OBJ_MAX_WEIGHTED_POWER ? dd_gt(fb, fthr) : dd_lt(fb, fthr)) k = pix;
        }
      }
    }
    ++round;
    if (s_fail) {
      failed = true;
      break;
    }
    tick(1);
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
          if (!setup_sweep(s)) { failed = true; break; }
          __syncthreads();
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
    // ---- fetch, in parallel: the winner's record, beta_i = alpha_i x_i[k], W_lo(k, own).
    //      Warps 0, 5, 6 and 7 (four sub-partitions) each read the record with one
    //      load per lane (lane l: word l) and share the FP64 bookkeeping:
    //      0: pivot and f, 5: S(new), 6: FP32 copy of alpha, 7: trace (CTA 0).
    if (warp == 0 || (warp >= 5 && warp <= 7)) {
      const unsigned long long* rw =
          reinterpret_cast<const unsigned long long*>(mrec_at(a, par, owner_of(k, n, P)));
      constexpr int kWords = (int)(sizeof(MixRecord) / 8);
      static_assert(kWords <= 32, "one record word per lane");
      const unsigned long long wv = lane < kWords ? rw[lane] : 0ull;
      auto word = [&](int i) {  // word i of the record as a double-word
        const unsigned long long u = __shfl_sync(0xffffffffu, wv, i);
        return dd{__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32))};
      };
      constexpr int oF = offsetof(MixRecord, f_new) / 8, oA = offsetof(MixRecord, alpha) / 8;
      constexpr int oC = offsetof(MixRecord, coef) / 8, oT = offsetof(MixRecord, Tk) / 8;
      const cdd al = cdd{word(oA), word(oA + 1)}, co = cdd{word(oC), word(oC + 1)};
      const dd fnew = word(oF);
      cdd tk = cdd_of(0.0f, 0.0f);  // lane p < n_o: row p of T' at pixel k
#pragma unroll
      for (int p = 0; p < kMaxPorts; ++p) {
        const cdd v = cdd{word(oT + 2 * p), word(oT + 2 * p + 1)};
        if (lane == p) tk = v;
      }
      if (warp == 0) {
        if (lane < n_o) s_pv.Tk[lane] = tk;
        if (lane == 0) {
          s_pv.k = k;
          s_pv.alpha = al;
          s_pv.coef = co;
          s_f = fnew;
          s_fthr = improve_bound<OBJ>(fnew, s_tau);
          s_bad = !isfinite(fnew.hi);
        }
      } else if (warp == 5) {
        // S(new) exactly as the scorer formed it
        if (lane < n_o) s_S[lane] = cdd_fma(co, tk, s_S[lane]);
      } else if (warp == 6) {
        if (lane == 0) s_alpha[r] = make_float2(al.re.hi, al.im.hi);  // alpha rounded to FP32
      } else if (cta == 0 && lane == 0) {
        // warp 7: the trace and alpha as double-words, converted to FP64 off the
        // chain (alpha before the next fold, the objectives at the end)
        if (n_acc < a.trace_cap) {
          if (a.trace) {
            int32_t* tr = a.trace + 4 * n_acc;
            tr[0] = a.mode == PNGF_FIRST_IMPROVEMENT ? s : (int)n_acc;
            tr[1] = pos_k;
            tr[2] = k;
            tr[3] = 0;
          }
          if (a.trace_f) *reinterpret_cast<dd*>(a.trace_f + n_acc) = fnew;
        }
        reinterpret_cast<cdd*>(a.xadd)[r] = al;
      }
    } else if (tid >= 32 && tid < 32 + r) {
      const int i = tid - 32;
      const float2 al = s_alpha[i], x = a.X[(size_t)k * R + i];
      s_beta[i] = make_float2(fmaf(al.x, x.x, -al.y * x.y), fmaf(al.x, x.y, al.y * x.x));
    } else if (tid >= 256 && tid < 256 + own) {
      const int jl = tid - 256, j = pb + jl;
      const size_t o = (size_t)min(k, j) * a.ldl + max(k, j);  // upper triangle of the symmetric W_lo
      s_wk[jl] = make_float2(a.Wr[o], a.Wi[o]);
    }
    __syncthreads();
    tick(2);
    // ---- keep the flip of pixel k
    if (s_bad) status = PNGF_ENUMERIC;
    if (n_acc >= a.trace_cap && status == PNGF_OK) status = PNGF_ECAPACITY;
    if (a.mode == PNGF_FIRST_IMPROVEMENT) {
      n_evals += pos_k - t + 1;
      t = pos_k + 1;
    } else {
      n_evals += n;
      ++sweeps_done;
    }
    ++acc_in_sweep;
    ++n_acc;
    // U2: the delayed sums sum_i beta_i x_i[j] in FP32.  Own pixels in blocks of
    // 32 (lane = pixel, consecutive words); the delayed columns split over
    // `parts` warps per block, whose partial sums meet in shared memory.
    {
      const int nb = (own + 31) >> 5;
      const int parts = min(kPartsMax, (kThreads / 32) / nb);  // nb * parts <= the CTA's warps
      if (warp < nb * parts) {
        const int jl = (warp % nb) * 32 + lane, part = warp / nb;
        float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
        if (jl < own) {
          int i = part;
          for (; i + parts < r; i += 2 * parts) {
            const float2 b0 = s_beta[i], x0 = Xs[i * OS + jl];
            const float2 b1 = s_beta[i + parts], x1 = Xs[(i + parts) * OS + jl];
            ax = fmaf(b0.x, x0.x, fmaf(-b0.y, x0.y, ax));
            ay = fmaf(b0.x, x0.y, fmaf(b0.y, x0.x, ay));
            bx = fmaf(b1.x, x1.x, fmaf(-b1.y, x1.y, bx));
            by = fmaf(b1.x, x1.y, fmaf(b1.y, x1.x, by));
          }
          if (i < r) {
            const float2 b0 = s_beta[i], x0 = Xs[i * OS + jl];
            ax = fmaf(b0.x, x0.x, fmaf(-b0.y, x0.y, ax));
            ay = fmaf(b0.x, x0.y, fmaf(b0.y, x0.x, ay));
          }
          s_part[part * OSS + jl] = make_float2(ax + bx, ay + by);
        }
      }
      __syncthreads();
      // c_j = W_lo(k, j) + delayed sum in FP32, promoted; alpha c_j in FP64; the
      // column is appended to the delayed set (one thread per own pixel)
      if (tid < own) {
        const int jl = tid;
        float sx = s_wk[jl].x, sy = s_wk[jl].y, dx = 0.f, dy = 0.f;
        for (int q = 0; q < parts; ++q) {
          dx += s_part[q * OSS + jl].x;
          dy += s_part[q * OSS + jl].y;
        }
        const float2 cf = make_float2(sx + dx, sy + dy);
        s_c[jl] = cf;
        s_ac[jl] = cdd_mul_cf(s_pv.alpha, cf.x, cf.y);
        const int j = pb + jl;
        Xs[r * OS + jl] = cf;
        a.X[(size_t)j * R + r] = cf;
        if (j == k) {
          const unsigned char nb2 = s_b[jl] ^ 1;
          s_b[jl] = nb2;
          a.b[j] = nb2;
          a.v[j] = nb2 ? s_dv[jl] : mk(0.0, 0.0);
        }
      }
    }
    __syncthreads();
    tick(13);
    // U3: one complex FMA per pixel and quantity q (0: diag, 1: e, 2 + p: row p
    // of T'), the quantities on warps of different sub-partitions
    {
      const int nq = 2 + n_o;
      for (int q = warp & 3; q < nq; q += 4)
        for (int jl = (warp >> 2) * 32 + lane; jl < own; jl += kThreads / 4) {
          if (q == 0) {
            s_diag[jl] = cdd_add(s_diag[jl], cdd_mul_cf(s_ac[jl], s_c[jl].x, s_c[jl].y));
          } else if (q == 1) {
            s_e[jl] = cdd_add(s_e[jl], cdd_mul_cf(s_pv.coef, s_c[jl].x, s_c[jl].y));
          } else {
            cdd* tq = s_T + (q - 2) * OSS + jl;
            *tq = cdd_fma(s_ac[jl], s_pv.Tk[q - 2], *tq);
          }
        }
    }
    __syncthreads();
    ++r;
    ++since_refresh;
    tick(4);
    if (r == R) {
      if (!flush()) { failed = true; break; }
      tick(3);
      if (a.refresh_k > 0 && since_refresh >= a.refresh_k) {
        since_refresh = 0;
        ++n_refresh;
        store_et(false);
        __syncthreads();
        // the delayed set is empty here: its shared memory holds the active-pixel
        // list, then the staging of the correction
        int* act = reinterpret_cast<int*>(work);
        const int m_act = active_list(a, act);
        sum_active += m_act;
        if (cta == 0)  // for the correction, after the next grid barrier
          for (int q = tid; q < m_act; q += blockDim.x) a.actg[q] = act[q];
        refresh_x_df(a, pb, pe, act, m_act);
        if (!grid_sync(ctl)) { failed = true; break; }
        tick(8);
        // the residual's copy ring after the list
        refresh_residual_df(a, pb, pe, act, m_act, work + rd_list_bytes(n), (unsigned)(kMixedWork - rd_list_bytes(n)));
        if (!grid_sync(ctl)) { failed = true; break; }
        // the accuracy guard of any CTA ends the search in every CTA (read after the barrier)
        if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EACCURACY) {
          status = PNGF_EACCURACY;
          break;
        }
        tick(9);
        correct_balanced(a, a.actg, m_act, reinterpret_cast<float*>(work), (int)(dynamic_smem_bytes() - state_bytes));
        if (!grid_sync(ctl)) { failed = true; break; }
        correct_combine(a, pb, pe);
        __syncthreads();
        tick(10);
        ports_partial(a, pb, pe);
        if (!grid_sync(ctl)) { failed = true; break; }
        tick(11);
        load_et();
        ports_total(a, s_o);
        if (tid < n_o) s_S[tid] = cdd_from(cmul(csub(s_o[tid], s_op.off[tid]), s_op.scale[tid]));
        if (tid == 32) {
          const double f = objective_of(s_op, s_o), thr = accept_threshold(s_op, f);
          s_f = dd_from(f);
          s_fthr = dd_from(OBJ == PNGF_OBJ_MAX_WEIGHTED_POWER ? f + thr : f - thr);
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
        if (!setup_sweep(s)) { failed = true; break; }
        __syncthreads();
      }
    }
  }
  __syncthreads();
  store_et(true);
  alpha_to_fp64();
  if (cta == 0 && a.trace_f)  // the objectives of the trace, kept as double-words
    for (long long i = tid; i < n_acc && i < a.trace_cap; i += blockDim.x)
      a.trace_f[i] = dd_to(*reinterpret_cast<const dd*>(a.trace_f + i));
  if (a.tensor_fold) tc_teardown(tcs, failed);  // after a failure: bounded wait for what was issued
  if (cta == 0 && threadIdx.x == 0) {
    if (failed) status = PNGF_ETIMEOUT;
    FOR_PORTS(p, n_o) ctl->o[p] = cadd(cmul(cdd_to(s_S[p]), s_iscale[p]), s_op.off[p]);
    ctl->f = dd_to(s_f);
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
    ctl->counters[7] = sum_active;
    ph[7] = clock64() - t_begin;
    for (int q = 0; q < 16; ++q) ctl->phase_cycles[q] = ph[q];
    if (a.counters)
      for (int q = 0; q < 8; ++q) a.counters[q] = ctl->counters[q];
    if (status == PNGF_ENUMERIC || status == PNGF_ETIMEOUT || status == PNGF_EINVAL || status == PNGF_EACCURACY)
      latch_status(ctl, status);
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


static void* mixed_kernel_for(int objective) {
  return objective == PNGF_OBJ_MAX_WEIGHTED_POWER ? (void*)dbs_mixed_kernel<PNGF_OBJ_MAX_WEIGHTED_POWER>
                                                  : (void*)dbs_mixed_kernel<PNGF_OBJ_MIN_INSERTION_LOSS>;
}

// dynamic shared memory of a launch: the own state of its largest CTA share, then the work area
static size_t mixed_smem(const pngf_ctx* c, int grid) {
  return own_state_bytes(c->cfg.n_o, own_stride(c->cfg.n_d, grid)) + kMixedWork;
}

static int mixed_grid(pngf_ctx* c) {
  static bool attr = false;
  if (!attr) {  // room for the largest own state (8 ports, kOwnMax pixels per CTA)
    const int most = (int)(own_state_bytes(kMaxPorts, kOwnMax) + kMixedWork);
    cudaFuncSetAttribute(dbs_mixed_kernel<PNGF_OBJ_MAX_WEIGHTED_POWER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         most);
    cudaFuncSetAttribute(dbs_mixed_kernel<PNGF_OBJ_MIN_INSERTION_LOSS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         most);
    cudaFuncSetAttribute(flush_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFlushSmem);
    attr = true;
  }
  // one CTA per SM: the work area alone is more than half of an SM's shared memory
  int g = c->n_sm;
  if (c->cfg.n_ctas > 0 && c->cfg.n_ctas < g) g = c->cfg.n_ctas;
  if (g > c->L.n_part) g = c->L.n_part;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mixed_kernel_for(c->cfg.objective), kThreads,
                                                mixed_smem(c, g));
  return per_sm >= 1 ? g : 0;
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
  int grid = mixed_grid(c);
  if (grid < 1) return PNGF_EINVAL;  // the own state does not fit in shared memory
  if ((c->cfg.n_d + grid - 1) / grid > kOwnMax) return PNGF_EINVAL;  // own-pixel state is shared memory
  // the delayed rows of the own pixels and the delayed sum's partials fit in the work area
  if (delayed_rows_bytes(a.R, own_stride(c->cfg.n_d, grid)) > kMixedWork) return PNGF_EINVAL;
  {  // the refresh residual's copy ring takes one list entry per group and stage at least, after the active list
    const int own = (c->cfg.n_d + grid - 1) / grid;
    const size_t list = rd_list_bytes(c->cfg.n_d);
    if (list + (size_t)kThreads * 16 > kMixedWork ||
        rd_rows(own, 1 + c->cfg.n_o, kThreads, (unsigned)(kMixedWork - list)) < 1)
      return PNGF_EINVAL;
  }
  cudaError_t err = cudaMemsetAsync(&ctl->bar_count, 0, 2 * sizeof(unsigned), c->stream);
  if (err != cudaSuccess) return PNGF_ECUDA;
  err = cudaMemsetAsync(a.slots, 0, (size_t)2 * grid * kSlotStride * sizeof(unsigned long long), c->stream);
  if (err != cudaSuccess) return PNGF_ECUDA;
  void* params[] = {&a};
  err = cudaLaunchCooperativeKernel(mixed_kernel_for(c->cfg.objective), dim3(grid), dim3(kThreads), params,
                                    mixed_smem(c, grid), c->stream);
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
