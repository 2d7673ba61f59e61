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

#include "pngf_internal.cuh"

namespace pngf {
namespace {

constexpr int kThreads = 512;
constexpr unsigned long long kSpinLimit = 1ull << 24;  // ~seconds with the 128 ns back-off

struct SweepArgs {
  int n, n_o, ldw, ldt;
  int mode, n_sweeps, trace_cap, refresh_k;
  const int* order;
  c128* W;
  c128* diag;
  c128* e;
  c128* T;
  c128* v;
  const c128* dv;
  uint8_t* b;
  int* pos_of;
  long long* part_key;  // [2][P]
  double* part_gain;    // [2][P]
  c128* cbuf;           // n
  c128* rbuf;           // (1 + n_o) x n
  c128* opart;          // P x n_o
  Control* ctl;
  int32_t* trace;
  double* trace_f;
  int64_t* counters;
  const c128* G;
  const c128* God;
  const c128* cd;
  const c128* co;
  ObjParams op;
};

// ---------------------------------------------------------------- grid barrier
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

__device__ bool grid_sync(Control* ctl) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned g = ld_volatile(&ctl->bar_gen);
    __threadfence();
    unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      unsigned long long it = 0;
      while (ld_volatile(&ctl->bar_gen) == g) {
        if (++it > kSpinLimit) {
          latch_status(ctl, PNGF_ETIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_ETIMEOUT) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------- block reductions
__device__ long long block_min_ll(long long x) {
  __shared__ long long sh[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) x = min(x, __shfl_down_sync(0xffffffffu, x, off));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    x = lane < (int)(blockDim.x >> 5) ? sh[lane] : LLONG_MAX;
    for (int off = 16; off > 0; off >>= 1) x = min(x, __shfl_down_sync(0xffffffffu, x, off));
    if (lane == 0) sh[0] = x;
  }
  __syncthreads();
  return sh[0];
}

// (gain, pixel): larger gain wins, ties -> lower pixel
__device__ __forceinline__ bool better(double g1, int p1, double g2, int p2) {
  return g1 > g2 || (g1 == g2 && p1 < p2);
}

__device__ void block_best(double& g, int& p) {
  __shared__ double shg[kThreads / 32];
  __shared__ int shp[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    double og = __shfl_down_sync(0xffffffffu, g, off);
    int op = __shfl_down_sync(0xffffffffu, p, off);
    if (better(og, op, g, p)) { g = og; p = op; }
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { shg[w] = g; shp[w] = p; }
  __syncthreads();
  if (w == 0) {
    g = lane < (int)(blockDim.x >> 5) ? shg[lane] : -INFINITY;
    p = lane < (int)(blockDim.x >> 5) ? shp[lane] : INT_MAX;
    for (int off = 16; off > 0; off >>= 1) {
      double og = __shfl_down_sync(0xffffffffu, g, off);
      int op = __shfl_down_sync(0xffffffffu, p, off);
      if (better(og, op, g, p)) { g = og; p = op; }
    }
    if (lane == 0) { shg[0] = g; shp[0] = p; }
  }
  __syncthreads();
  g = shg[0];
  p = shp[0];
}

// ---------------------------------------------------------------- scoring
// Candidate objective for flipping pixel j against the current state (Eq. 14).
// Returns false for a numerically singular candidate (|d_j| < 1e-14).
__device__ __forceinline__ bool score_pixel(const SweepArgs& a, const ObjParams& op, int j, const c128* o,
                                            double& f_new, c128* o_new) {
  c128 dvj = a.dv[j];
  c128 delta = a.b[j] ? mk(-dvj.x, -dvj.y) : dvj;
  c128 dj = csub(mk(1.0, 0.0), cmul(delta, a.diag[j]));
  if (cabs2(dj) < 1e-28) return false;
  c128 alpha = cdiv(delta, dj);
  c128 coef = cmul(alpha, a.e[j]);
  double fn = 0.0;
#pragma unroll 1
  for (int p = 0; p < a.n_o; ++p) {
    c128 on = cfma(coef, a.T[(size_t)p * a.ldt + j], o[p]);
    if (o_new) o_new[p] = on;
    fn += objective_term(op, p, on);
  }
  f_new = fn;
  return true;
}

// packed upper-triangle index -> (row, column); off(i) = i*n - i*(i-1)/2
__device__ __forceinline__ void tri_rc(long long e, int n, int& i, int& j) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    long long off = (long long)mid * n - (long long)mid * (mid - 1) / 2;
    if (off <= e) lo = mid; else hi = mid - 1;
  }
  i = lo;
  j = lo + (int)(e - ((long long)lo * n - (long long)lo * (lo - 1) / 2));
}

// W += alpha c c^T on packed elements [eb, ee) of the upper triangle.
// Thread t walks elements eb + t + m*blockDim; four consecutive steps of the
// walk are issued together so that four independent loads are in flight.
__device__ __forceinline__ void tri_step(int& i, int& j, int n, int stride) {
  j += stride;
  // carry into the following rows (row i+1 starts at column i+1); past the
  // last row the walk is beyond ee and the caller stops
  while (j >= n && i < n) {
    j -= n;
    ++i;
    j += i;
  }
}

__device__ void rank1_upper(c128* __restrict__ W, int n, int ldw, const c128* __restrict__ c, c128 alpha,
                            long long eb, long long ee) {
  long long e = eb + threadIdx.x;
  if (e >= ee) return;
  const int stride = blockDim.x;
  int i0, j0;
  tri_rc(e, n, i0, j0);
  while (e + 3LL * stride < ee) {
    int i1 = i0, j1 = j0;
    tri_step(i1, j1, n, stride);
    int i2 = i1, j2 = j1;
    tri_step(i2, j2, n, stride);
    int i3 = i2, j3 = j2;
    tri_step(i3, j3, n, stride);
    c128* p0 = W + (size_t)i0 * ldw + j0;
    c128* p1 = W + (size_t)i1 * ldw + j1;
    c128* p2 = W + (size_t)i2 * ldw + j2;
    c128* p3 = W + (size_t)i3 * ldw + j3;
    c128 w0 = *p0, w1 = *p1, w2 = *p2, w3 = *p3;
    c128 c0 = c[j0], c1 = c[j1], c2 = c[j2], c3 = c[j3];
    c128 a0 = cmul(alpha, c[i0]);
    c128 a1 = (i1 == i0) ? a0 : cmul(alpha, c[i1]);
    c128 a2 = (i2 == i1) ? a1 : cmul(alpha, c[i2]);
    c128 a3 = (i3 == i2) ? a2 : cmul(alpha, c[i3]);
    *p0 = cfma(a0, c0, w0);
    *p1 = cfma(a1, c1, w1);
    *p2 = cfma(a2, c2, w2);
    *p3 = cfma(a3, c3, w3);
    i0 = i3;
    j0 = j3;
    tri_step(i0, j0, n, stride);
    e += 4LL * stride;
  }
  for (; e < ee; e += stride) {
    c128* p = W + (size_t)i0 * ldw + j0;
    *p = cfma(cmul(alpha, c[i0]), c[j0], *p);
    tri_step(i0, j0, n, stride);
  }
}

struct Pivot {
  int k;
  c128 alpha, coef;  // coef = alpha e_k
  c128 Tk[kMaxPorts];
};

__device__ __forceinline__ void make_pivot(const SweepArgs& a, int k, Pivot& pv) {
  c128 dvk = a.dv[k];
  c128 delta = a.b[k] ? mk(-dvk.x, -dvk.y) : dvk;
  c128 dk = csub(mk(1.0, 0.0), cmul(delta, a.diag[k]));
  pv.k = k;
  pv.alpha = cdiv(delta, dk);
  pv.coef = cmul(pv.alpha, a.e[k]);
  FOR_PORTS(p, a.n_o) pv.Tk[p] = a.T[(size_t)p * a.ldt + k];
}

// state update of pixels [pb, pe) given c = cbuf
__device__ void update_state(const SweepArgs& a, const Pivot& pv, int pb, int pe) {
  for (int j = pb + threadIdx.x; j < pe; j += blockDim.x) {
    c128 cj = a.cbuf[j];
    c128 aj = cmul(pv.alpha, cj);
    a.diag[j] = cfma(aj, cj, a.diag[j]);
    a.e[j] = cfma(pv.coef, cj, a.e[j]);
#pragma unroll 1
    for (int p = 0; p < a.n_o; ++p) {
      c128* t = a.T + (size_t)p * a.ldt + j;
      *t = cfma(aj, pv.Tk[p], *t);
    }
    if (j == pv.k) {
      uint8_t nb = a.b[j] ^ 1;
      a.b[j] = nb;
      a.v[j] = nb ? a.dv[j] : mk(0.0, 0.0);
    }
  }
}

// c_j = W[k][j] (j >= k) or W[j][k] (j < k) for j in [pb, pe)
__device__ void gather_column(const SweepArgs& a, int k, int pb, int pe) {
  for (int j = pb + threadIdx.x; j < pe; j += blockDim.x)
    a.cbuf[j] = (j >= k) ? a.W[(size_t)k * a.ldw + j] : a.W[(size_t)j * a.ldw + k];
}

// ---------------------------------------------------------------- refresh
// One FP64 iterative-refinement step of e and of the rows of T:
//   e: r = c_d - (e - G (v.e)),         e += r + W (v.r)
//   T: R = G_od - (T - (T diag v) G),   T += R + (R diag v) W      (G, W symmetric)
// Scratch rbuf holds four blocks of nv = 1 + n_o vectors of length n:
//   [0] residuals r, [1] x = v.[e, T], [2] x2 = v.r, [3] row sums of the upper triangle.
__device__ __forceinline__ c128* rvec(const SweepArgs& a, int blk, int q) {
  return a.rbuf + ((size_t)blk * (1 + a.n_o) + q) * a.n;
}

__device__ __forceinline__ c128 warp_sum(c128 v) {
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// R0: x = v.[e, T] for own pixels
__device__ void refresh_x(const SweepArgs& a, int pb, int pe) {
  for (int j = pb + threadIdx.x; j < pe; j += blockDim.x) {
    c128 vj = a.v[j];
    rvec(a, 1, 0)[j] = cmul(vj, a.e[j]);
    for (int p = 0; p < a.n_o; ++p) rvec(a, 1, 1 + p)[j] = cmul(vj, a.T[(size_t)p * a.ldt + j]);
  }
}

// R1: residuals of own rows (row j of G dotted with x), and x2 = v.r
#define FOR_VECS(q, nv) _Pragma("unroll") for (int q = 0; q < 1 + kMaxPorts; ++q) if (q < (nv))
__device__ __noinline__ void refresh_residual(const SweepArgs& a, int pb, int pe) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nv = 1 + a.n_o;
  for (int j = pb + warp; j < pe; j += nw) {
    const c128* g = a.G + (size_t)j * a.n;
    c128 acc[1 + kMaxPorts];
    FOR_VECS(q, nv) acc[q] = mk(0.0, 0.0);
#pragma unroll 4
    for (int i = lane; i < a.n; i += 32) {
      c128 gi = g[i];
      FOR_VECS(q, nv) acc[q] = cfma(gi, rvec(a, 1, q)[i], acc[q]);
    }
    FOR_VECS(q, nv) {
      c128 sum = warp_sum(acc[q]);
      if (lane == 0) {
        c128 rhs = q == 0 ? a.cd[j] : a.God[(size_t)(q - 1) * a.n + j];
        c128 y = q == 0 ? a.e[j] : a.T[(size_t)(q - 1) * a.ldt + j];
        c128 r = cadd(csub(rhs, y), sum);
        rvec(a, 0, q)[j] = r;
        rvec(a, 2, q)[j] = cmul(a.v[j], r);
      }
    }
  }
}

// R2: corrections (I + W V) r for own rows, W symmetric with its upper
// triangle current: row j takes sum_{i>=j} W[j][i] x2_i from its own row and
// sum_{i<j} W[i][j] x2_i from the rows above (a strip of columns [pb, pe)).
// The residual r is FP64; the product W x2 only has to be accurate relative
// to |r| (classic mixed-precision iterative refinement), so it runs in FP32
// arithmetic on the FP64-stored W and is added to r in FP64.
struct f2c {
  float x, y;
};
__device__ __forceinline__ f2c f2(c128 a) { return f2c{(float)a.x, (float)a.y}; }
__device__ __forceinline__ f2c f2fma(f2c a, f2c b, f2c c) {
  return f2c{fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y))};
}
__device__ __forceinline__ f2c f2sum(f2c v) {
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

__device__ __noinline__ void refresh_correct(const SweepArgs& a, int pb, int pe) {
  __shared__ f2c red[kThreads / 32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nv = 1 + a.n_o;
  // upper part, one warp per own row
  for (int j = pb + warp; j < pe; j += nw) {
    const c128* w = a.W + (size_t)j * a.ldw;
    f2c acc[1 + kMaxPorts];
    FOR_VECS(q, nv) acc[q] = f2c{0.f, 0.f};
#pragma unroll 4
    for (int i = j + lane; i < a.n; i += 32) {
      f2c wi = f2(w[i]);
      FOR_VECS(q, nv) acc[q] = f2fma(wi, f2(rvec(a, 2, q)[i]), acc[q]);
    }
    FOR_VECS(q, nv) {
      f2c sum = f2sum(acc[q]);
      if (lane == 0) rvec(a, 3, q)[j] = mk(sum.x, sum.y);
    }
  }
  __syncthreads();
  // lower part: columns of this CTA in chunks of 32, rows above spread over warps
  for (int c0 = pb; c0 < pe; c0 += 32) {
    const int j = c0 + lane;
    const int rows = min(pe, c0 + 32) - 1;  // rows i < j <= rows
    f2c acc[1 + kMaxPorts];
    FOR_VECS(q, nv) acc[q] = f2c{0.f, 0.f};
#pragma unroll 4
    for (int i = warp; i < rows; i += nw) {
      if (i < j && j < pe) {
        f2c wij = f2(a.W[(size_t)i * a.ldw + j]);
        FOR_VECS(q, nv) acc[q] = f2fma(wij, f2(rvec(a, 2, q)[i]), acc[q]);
      }
    }
    for (int q = 0; q < nv; ++q) {
      f2c mine = f2c{0.f, 0.f};
      FOR_VECS(qq, nv) if (qq == q) mine = acc[qq];
      red[warp][lane] = mine;
      __syncthreads();
      if (warp == 0 && j < pe) {
        double lx = 0.0, ly = 0.0;
        for (int w2 = 0; w2 < nw; ++w2) {
          lx += red[w2][lane].x;
          ly += red[w2][lane].y;
        }
        c128 d = cadd(rvec(a, 0, q)[j], cadd(rvec(a, 3, q)[j], mk(lx, ly)));
        if (q == 0) {
          a.e[j] = cadd(a.e[j], d);
        } else {
          c128* t = a.T + (size_t)(q - 1) * a.ldt + j;
          *t = cadd(*t, d);
        }
      }
      __syncthreads();
    }
  }
}

// partial o sums of pixels [pb, pe) -> opart[cta]
__device__ __noinline__ void ports_partial(const SweepArgs& a, int pb, int pe) {
  __shared__ c128 red[kMaxPorts][kThreads / 32];
  c128 acc[kMaxPorts];
  FOR_PORTS(p, a.n_o) acc[p] = mk(0.0, 0.0);
  for (int j = pb + threadIdx.x; j < pe; j += blockDim.x) {
    c128 ve = cmul(a.v[j], a.e[j]);
    FOR_PORTS(p, a.n_o) acc[p] = cfma(a.God[(size_t)p * a.n + j], ve, acc[p]);
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  FOR_PORTS(p, a.n_o) {
    for (int off = 16; off > 0; off >>= 1) {
      acc[p].x += __shfl_down_sync(0xffffffffu, acc[p].x, off);
      acc[p].y += __shfl_down_sync(0xffffffffu, acc[p].y, off);
    }
  }
  __syncthreads();
  if (lane == 0) {
    FOR_PORTS(p, a.n_o) red[p][w] = acc[p];
  }
  __syncthreads();
  if (threadIdx.x < a.n_o) {
    c128 s = mk(0.0, 0.0);
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s = cadd(s, red[threadIdx.x][q]);
    a.opart[(size_t)blockIdx.x * a.n_o + threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------- persistent DBS
__global__ void __launch_bounds__(kThreads) dbs_fp64_kernel(SweepArgs a) {
  const int P = gridDim.x, cta = blockIdx.x;
  const int n = a.n;
  const int pb = (int)((long long)n * cta / P), pe = (int)((long long)n * (cta + 1) / P);
  const long long E = (long long)n * (n + 1) / 2;
  const long long eb = E * cta / P, ee = E * (cta + 1) / P;
  Control* ctl = a.ctl;
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
  long long n_acc = 0, n_evals = 0, n_refresh = 0;
  int sweeps_done = 0, converged = 0, status = PNGF_OK;
  // per-phase SM-cycle accounting of CTA 0 (thread 0 sees every phase boundary)
  const bool timer = (cta == 0 && threadIdx.x == 0);
  long long ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long t_last = clock64(), t_begin = t_last;
  auto tick = [&](int phase) {
    if (timer) {
      long long now = clock64();
      ph[phase] += now - t_last;
      t_last = now;
    }
  };
  int since_refresh = ctl->since_refresh;
  int s = 0, t = 0, acc_in_sweep = 0, slot = 0;
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
  }
  const long long max_steps = a.n_sweeps;  // BEST mode: one kept flip per step
  while (!failed) {
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
      if (threadIdx.x == 0) a.part_key[slot * P + cta] = best;
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
        long long best = LLONG_MAX;
        for (int q = lane; q < P; q += 32) best = min(best, a.part_key[slot * P + q]);
        for (int off = 16; off > 0; off >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, off));
        if (best != LLONG_MAX) {
          pos_k = (int)best;
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
    const int k = s_k, pos_k = s_pos;
    if (k == -2 || *reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) {
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
    gather_column(a, k, pb, pe);
    tick(2);
    if (!grid_sync(ctl)) { failed = true; break; }
    tick(3);
    update_state(a, s_pv, pb, pe);
    rank1_upper(a.W, n, a.ldw, a.cbuf, s_pv.alpha, eb, ee);
    __syncthreads();
    tick(4);
    ++since_refresh;
    if (a.refresh_k > 0 && since_refresh >= a.refresh_k) {
      since_refresh = 0;
      ++n_refresh;
      if (!grid_sync(ctl)) { failed = true; break; }
      refresh_x(a, pb, pe);
      if (!grid_sync(ctl)) { failed = true; break; }
      refresh_residual(a, pb, pe);
      if (!grid_sync(ctl)) { failed = true; break; }
      refresh_correct(a, pb, pe);
      if (!grid_sync(ctl)) { failed = true; break; }
      ports_partial(a, pb, pe);
      if (!grid_sync(ctl)) { failed = true; break; }
      if (threadIdx.x == 0) {
        FOR_PORTS(p, a.n_o) {
          c128 acc = mk(0.0, 0.0);
          for (int q = 0; q < P; ++q) acc = cadd(acc, a.opart[(size_t)q * a.n_o + p]);
          s_o[p] = cadd(a.co[p], acc);
        }
        s_f = objective_of(s_op, s_o);
      }
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
    ctl->counters[7] = 0;
    ph[7] = clock64() - t_begin;
    for (int q = 0; q < 8; ++q) ctl->phase_cycles[q] = ph[q];
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

SweepArgs make_args(pngf_ctx* c) {
  SweepArgs a{};
  const Layout& L = c->L;
  a.n = c->cfg.n_d;
  a.n_o = c->cfg.n_o;
  a.ldw = L.ldw;
  a.ldt = L.ldt;
  a.mode = c->cfg.mode;
  a.refresh_k = c->cfg.refresh_k;
  a.W = at<c128>(c, L.W);
  a.diag = at<c128>(c, L.diag);
  a.e = at<c128>(c, L.e);
  a.T = at<c128>(c, L.T);
  a.v = at<c128>(c, L.v);
  a.dv = c->dv;
  a.b = at<uint8_t>(c, L.b);
  a.pos_of = at<int>(c, L.pos_of);
  a.part_key = at<long long>(c, L.part);
  a.part_gain = reinterpret_cast<double*>(a.part_key + 2 * L.n_part);
  a.opart = reinterpret_cast<c128*>(a.part_gain + 2 * L.n_part);
  a.cbuf = at<c128>(c, L.cbuf);
  a.rbuf = at<c128>(c, L.rbuf);
  a.ctl = at<Control>(c, L.ctl);
  a.G = c->G;
  a.God = c->God;
  a.cd = c->cd;
  a.co = c->co;
  a.op = c->obj;
  return a;
}

}  // namespace

int sweep_grid_size(pngf_ctx* c) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dbs_fp64_kernel, kThreads, 0);
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
  int grid = c->coop_ctas;
  void* params[] = {&a};
  err = cudaLaunchCooperativeKernel((const void*)dbs_fp64_kernel, dim3(grid), dim3(kThreads), params, 0,
                                    c->stream);
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

}  // namespace pngf
