// Device building blocks shared by the FP64 and mixed-precision DBS kernels
// (scoring, selection, pivot, state update, grid barrier, FP64 refresh).
// Included by sweep.cu and sweep_mixed.cu; everything has internal linkage.
#pragma once

#include "pngf_internal.cuh"

namespace pngf {
namespace {

constexpr int kThreads = 512;
// Bound of every device-side wait on other CTAs: at most 2^24 polls (or a
// context's own count, Control::spin_limit, set by pngf_set_wait_limit) and
// at most kWaitNs of wall-clock time on the GPU's global timer, whichever
// comes first.  The time cap matters: a poll is an L2 round trip plus a short
// back-off, and under contention (every CTA of the grid polling one line) a
// poll can take far longer than the uncontended ~1 us, so a bound in polls
// alone can stretch to minutes.
constexpr unsigned long long kSpinLimit = 1ull << 24;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long spin_limit_of(const Control* ctl) {
  const unsigned long long l = *reinterpret_cast<const volatile unsigned long long*>(&ctl->spin_limit);
  return l ? l : kSpinLimit;
}

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
  const double* Gs;  // Re G + Im G
  const c128* God;
  const c128* cd;
  const c128* co;
  ObjParams op;
  // mixed path
  int mixed, ldl, R;
  int tensor_fold;        // mixed: fold the delayed set on the tensor cores
  unsigned char* tcimgA;  // operand images of the tensor-core fold
  unsigned char* tcimgB;
  float* Wr;  // planar FP32 copy of W (upper triangle current)
  float* Wi;
  float2* X;  // n x R delayed columns c_i in FP32 (row j holds c_0[j] .. c_{R-1}[j])
  c128* xa;   // R coefficients alpha_i
  void* rec;  // [2][P] candidate records
  unsigned long long* slots;  // [2][P] round words of the mixed search, 128 B apart
  int* actg;                  // n: active-pixel list of the last refresh (written by CTA 0)
  const float4* G2;           // n x n: G as FP32 pairs (Re hi, Im hi, Re lo, Im lo)
  float4* xs;                 // (1 + n_o) x n x 2: x = v.[e, T] at the active pixels, FP32 pairs, each part twice
  float4* xadd;               // R: alpha_i of the mixed search as double-word pairs, until copied to xa
};

// a CTA's candidate of one scoring round, with the state the pivot needs
struct CandRecord {
  long long key;  // FIRST: visiting position; BEST: unused (see gain)
  double gain;
  int pixel;
  int b;
  c128 alpha, coef;  // Sherman-Morrison coefficient of the flip and alpha * e_k
  c128 dv;
  c128 T[kMaxPorts];
};

// ---------------------------------------------------------------- grid barrier
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

// Acquire/release fence at GPU scope.  Paired with a relaxed store (release)
// or after a relaxed load (acquire) it orders exactly what the barrier and
// the word exchange need, and it is lighter than the sequentially consistent
// fence of __threadfence().
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Grid barrier on one monotonically increasing arrival counter (reset to 0
// before every launch): the arrival that returns `old` belongs to barrier
// old / P, which is complete once the counter reaches (old / P + 1) P.  One
// atomic per CTA and no generation word, so the last arrival releases the
// others without a further round trip.  The spin is bounded: on expiry the
// CTA latches PNGF_ETIMEOUT and returns false.
__device__ bool grid_sync(Control* ctl) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    fence_acq_rel_gpu();  // release: this CTA's writes before its arrival
    const unsigned P = gridDim.x;
    const unsigned long long lim = spin_limit_of(ctl);
    const unsigned old = atomicAdd(&ctl->bar_count, 1u);
    const unsigned target = (old / P + 1) * P;
    unsigned long long it = 0;
    const unsigned long long t0 = global_ns();
    while ((int)(ld_volatile(&ctl->bar_count) - target) < 0) {
      if (++it > lim || ((it & 63) == 0 && global_ns() - t0 > kWaitNs)) {
        latch_status(ctl, PNGF_ETIMEOUT);
        ok = 0;
        break;
      }
      if (it > 256) __nanosleep(32);
    }
    fence_acq_rel_gpu();  // acquire: every CTA's writes before the others' arrivals
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Test hook of the timeout path (pngf_set_wait_limit): CTA hold_cta - 1 waits
// on a flag that nothing sets, bounded by a longer wait than the others' own
// limit, before it takes part in anything grid-wide; the other CTAs' bounded
// waits for it run out and latch PNGF_ETIMEOUT.  One-shot: the hold is cleared.
__device__ void hold_if_asked(Control* ctl) {
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(&ctl->hold_cta) == (int)blockIdx.x + 1) {
    const unsigned long long lim = 4 * spin_limit_of(ctl), t0 = global_ns();
    for (unsigned long long it = 0; it < lim && global_ns() - t0 < 4 * kWaitNs; ++it) {
      if (*reinterpret_cast<volatile int*>(&ctl->hold_flag) != 0) break;
      __nanosleep(256);
    }
    ctl->hold_cta = 0;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- FIRST-mode selection cells
// Round rd of the search uses cell sel[rd % 3]: every CTA with a candidate
// atomically lowers it to (position << 10 | cta) before the round's barrier,
// and every CTA reads it after.  CTA 0 re-arms the cell of round rd + 1 during
// round rd: its last readers (round rd - 2) finished before barrier rd - 1,
// and its first writers (round rd + 1) start after barrier rd.
__device__ __forceinline__ void sel_offer(Control* ctl, int rd, long long pos, int cta) {
  if (pos != LLONG_MAX) atomicMin(&ctl->sel[rd % 3], ((unsigned long long)pos << 10) | (unsigned)cta);
  if (cta == 0) ctl->sel[(rd + 1) % 3] = ~0ull;
}

__device__ __forceinline__ unsigned long long sel_read(Control* ctl, int rd) {
  return *reinterpret_cast<volatile unsigned long long*>(&ctl->sel[rd % 3]);
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
                                            double& f_new, c128* o_new, c128* alpha_out = nullptr,
                                            c128* coef_out = nullptr) {
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
  if (alpha_out) {
    *alpha_out = alpha;
    *coef_out = coef;
  }
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

// block 2 holds x2 = v.r in FP32 (it only feeds the FP32 correction product)
__device__ __forceinline__ float2* x2f(const SweepArgs& a, int q) {
  return reinterpret_cast<float2*>(rvec(a, 2, 0)) + (size_t)q * a.n;
}

__device__ __forceinline__ c128 warp_sum(c128 v) {
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// Re x + Im x of the refined vectors, for the three-multiplication products of
// the residual (block 3 holds them until the correction overwrites it)
__device__ __forceinline__ double* xsum(const SweepArgs& a, int q) {
  return reinterpret_cast<double*>(rvec(a, 3, 0)) + (size_t)q * a.n;
}

// R0: x = v.[e, T] for own pixels
__device__ void refresh_x(const SweepArgs& a, int pb, int pe) {
  for (int j = pb + threadIdx.x; j < pe; j += blockDim.x) {
    c128 vj = a.v[j];
    const c128 x0 = cmul(vj, a.e[j]);
    rvec(a, 1, 0)[j] = x0;
    xsum(a, 0)[j] = x0.x + x0.y;
    for (int p = 0; p < a.n_o; ++p) {
      const c128 xp = cmul(vj, a.T[(size_t)p * a.ldt + j]);
      rvec(a, 1, 1 + p)[j] = xp;
      xsum(a, 1 + p)[j] = xp.x + xp.y;
    }
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// The refresh kernels carry the number of refined vectors NV = 1 + n_o as a
// template parameter: every loop over the vectors is then fully unrolled with
// no predicated-off FP64 work (the FP64 pipe is the scarce one on GB300).

// Ascending list of the pixels with b_i = 1 (the only nonzero entries of
// x = v.[e, T]) in shared memory act[0, m); returns m (the same in every thread).
__device__ int active_list(const SweepArgs& a, int* act) {
  __shared__ int s_scan[kThreads / 32];
  __shared__ int s_m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int chunk = (a.n + blockDim.x - 1) / blockDim.x;
  const int i0 = min(a.n, (int)threadIdx.x * chunk), i1 = min(a.n, i0 + chunk);
  int c = 0;
  for (int i = i0; i < i1; ++i) c += a.b[i] != 0;
  int incl = c;  // inclusive scan over the block, thread order = pixel order
  for (int off = 1; off < 32; off <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  __syncthreads();
  if (lane == 31) s_scan[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? s_scan[lane] : 0;
    for (int off = 1; off < 32; off <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < nw) s_scan[lane] = w;
    if (lane == nw - 1) s_m = w;
  }
  __syncthreads();
  int o = incl - c + (warp > 0 ? s_scan[warp - 1] : 0);
  for (int i = i0; i < i1; ++i)
    if (a.b[i]) act[o++] = i;
  __syncthreads();
  return s_m;
}

// number of entries of the ascending list act[0, m) below v (shared memory)
__device__ __forceinline__ int count_below(const int* act, int m, int v) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (act[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// R1: residuals of own rows (row j of G dotted with x), and x2 = v.r.  With
// act (shared memory, room for n entries) only the columns of G at pixels
// with b_i = 1 are visited: x vanishes elsewhere, so the FP64 work follows the
// number of "on" pixels instead of n.  Each complex product runs as Gauss's
// three real multiplications, (A + iB)(u + iw) = (Au - Bw) + i((A + B)(u + w)
// - Au - Bw), with A + B precomputed (Gs) and u + w from refresh_x: three FP64
// FMAs per element and vector instead of four.
template <int NV>
__device__ __noinline__ int refresh_residual_t(const SweepArgs& a, int pb, int pe, int* act) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int m = act ? active_list(a, act) : a.n;
  if (act && blockIdx.x == 0)  // for the correction, after the next grid barrier
    for (int t = threadIdx.x; t < m; t += blockDim.x) a.actg[t] = act[t];
  for (int j = pb + warp; j < pe; j += nw) {
    const c128* g = a.G + (size_t)j * a.n;
    const double* gs = a.Gs + (size_t)j * a.n;
    double p1[NV], p2[NV], p3[NV];  // A u, B w, (A + B)(u + w)
#pragma unroll
    for (int q = 0; q < NV; ++q) p1[q] = p2[q] = p3[q] = 0.0;
    auto madd = [&](int i) {
      const c128 gi = g[i];
      const double si = gs[i];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const c128 x = rvec(a, 1, q)[i];
        p1[q] = fma(gi.x, x.x, p1[q]);
        p2[q] = fma(gi.y, x.y, p2[q]);
        p3[q] = fma(si, xsum(a, q)[i], p3[q]);
      }
    };
    if (act) {
#pragma unroll 4
      for (int t = lane; t < m; t += 32) madd(act[t]);
    } else {
#pragma unroll 4
      for (int i = lane; i < a.n; i += 32) madd(i);
    }
    // lane q takes vector q's sums, then one code path finishes every vector
    double t1 = 0.0, t2 = 0.0, t3 = 0.0;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const double s1 = warp_sum_d(p1[q]), s2 = warp_sum_d(p2[q]), s3 = warp_sum_d(p3[q]);
      if (lane == q) {
        t1 = s1;
        t2 = s2;
        t3 = s3;
      }
    }
    if (lane < NV) {
      const int q = lane;
      const c128 sum = mk(t1 - t2, t3 - t1 - t2);
      const c128 rhs = q == 0 ? a.cd[j] : a.God[(size_t)(q - 1) * a.n + j];
      const c128 y = q == 0 ? a.e[j] : a.T[(size_t)(q - 1) * a.ldt + j];
      const c128 r = cadd(csub(rhs, y), sum);
      rvec(a, 0, q)[j] = r;
      const c128 x2 = cmul(a.v[j], r);
      x2f(a, q)[j] = make_float2((float)x2.x, (float)x2.y);
    }
  }
  return m;
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

// element (i, j) of the maintained W with i <= j, as FP32 (FP64 storage or the
// planar FP32 copy of the mixed path)
// (MIXED is a template parameter: a runtime test would leave the FP64
// path's conversions in the mixed loops as predicated-off FP64 instructions,
// which still occupy the FP64 pipe.)
template <bool MIXED>
__device__ __forceinline__ f2c w_upper(const SweepArgs& a, int i, int j) {
  if (MIXED) {
    size_t o = (size_t)i * a.ldl + j;
    return f2c{a.Wr[o], a.Wi[o]};
  }
  return f2(a.W[(size_t)i * a.ldw + j]);
}

// four consecutive elements W(j, i0 .. i0+3) of the maintained W as FP32
// (i0 % 4 == 0; rows are padded to a multiple of 4 so the read stays inside
// the row; elements past n are masked by the caller)
template <bool MIXED>
__device__ __forceinline__ void w_row4(const SweepArgs& a, int j, int i0, f2c w[4]) {
  if (MIXED) {
    const size_t o = (size_t)j * a.ldl + i0;
    const float4 re = *reinterpret_cast<const float4*>(a.Wr + o);
    const float4 im = *reinterpret_cast<const float4*>(a.Wi + o);
    w[0] = f2c{re.x, im.x};
    w[1] = f2c{re.y, im.y};
    w[2] = f2c{re.z, im.z};
    w[3] = f2c{re.w, im.w};
  } else {
    const c128* p = a.W + (size_t)j * a.ldw + i0;
#pragma unroll
    for (int u = 0; u < 4; ++u) w[u] = f2(p[u]);
  }
}

// R2, upper part: one warp per own row j, sum over i >= j of W[j][i] x2_i
// with four-wide row reads, four chunks in flight per lane.
template <int NV, bool MIXED>
__device__ __forceinline__ void correct_upper(const SweepArgs& a, int pb, int pe) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = a.n;
  for (int j = pb + warp; j < pe; j += nw) {
    f2c acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = f2c{0.f, 0.f};
    const int ib = j & ~3;
#pragma unroll 4
    for (int i0 = ib + 4 * lane; i0 < n; i0 += 128) {
      f2c w[4];
      w_row4<MIXED>(a, j, i0, w);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u;
        if (i >= j && i < n) {
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            const float2 x = x2f(a, q)[i];
            acc[q] = f2fma(w[u], f2c{x.x, x.y}, acc[q]);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      f2c sum = f2sum(acc[q]);
      if (lane == 0) rvec(a, 3, q)[j] = mk(sum.x, sum.y);
    }
  }
}

// R2: corrections (I + W V) r for own rows, W symmetric with its upper
// triangle current: row j takes sum_{i>=j} W[j][i] x2_i from its own row and
// sum_{i<j} W[i][j] x2_i from the rows above (a strip of columns [pb, pe)).
// The residual r is FP64; the product W x2 only has to be accurate relative
// to |r| (classic mixed-precision iterative refinement), so it runs in FP32
// arithmetic and is added to r in FP64.  x2 = v.r vanishes where b_i = 0, so
// with the active list act[0, m) only those rows of the strip are read.
template <int NV, bool MIXED>
__device__ __noinline__ void refresh_correct_t(const SweepArgs& a, int pb, int pe, const int* act, int m) {
  __shared__ f2c red[kThreads / 32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  correct_upper<NV, MIXED>(a, pb, pe);
  __syncthreads();
  // lower part: columns of this CTA in blocks of 32 (lane = column), the rows
  // above spread over the warps, eight rows in flight per warp
  int t_end;  // rows i < pe - 1 only (the active list is ascending)
  if (act) {
    int lo = 0, hi = m;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (act[mid] < pe - 1) lo = mid + 1; else hi = mid;
    }
    t_end = lo;
  } else {
    t_end = max(pe - 1, 0);
  }
  for (int c0 = pb; c0 < pe; c0 += 32) {
    const int j = c0 + lane;
    const bool colok = j < pe;
    f2c acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = f2c{0.f, 0.f};
    for (int t = warp; t < t_end; t += 8 * nw) {
      int ii[8];
      f2c w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int tu = t + u * nw;
        ii[u] = tu < t_end ? (act ? act[tu] : tu) : -1;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        w[u] = f2c{0.f, 0.f};
        if (ii[u] >= 0 && colok && ii[u] < j) w[u] = w_upper<MIXED>(a, ii[u], j);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (ii[u] >= 0 && colok && ii[u] < j) {
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            const float2 x = x2f(a, q)[ii[u]];
            acc[q] = f2fma(w[u], f2c{x.x, x.y}, acc[q]);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      red[warp][lane] = acc[q];
      __syncthreads();
      if (warp == 0 && colok) {
        double lx = 0.0, ly = 0.0;
        for (int w2 = 0; w2 < nw; ++w2) {
          lx += red[w2][lane].x;
          ly += red[w2][lane].y;
        }
        c128 d = cadd(rvec(a, 0, q)[j], cadd(rvec(a, 3, q)[j], mk(lx, ly)));
        if (q == 0) {
          a.e[j] = cadd(a.e[j], d);
        } else {
          c128* tq = a.T + (size_t)(q - 1) * a.ldt + j;
          *tq = cadd(*tq, d);
        }
      }
      __syncthreads();
    }
  }
}

// act: shared memory for n pixel indices, or nullptr (dense visit of all
// columns); returns the length of the active list (n when dense)
__device__ int refresh_residual(const SweepArgs& a, int pb, int pe, int* act = nullptr) {
  switch (a.n_o) {
    case 1: return refresh_residual_t<2>(a, pb, pe, act);
    case 2: return refresh_residual_t<3>(a, pb, pe, act);
    case 3: return refresh_residual_t<4>(a, pb, pe, act);
    case 4: return refresh_residual_t<5>(a, pb, pe, act);
    case 5: return refresh_residual_t<6>(a, pb, pe, act);
    case 6: return refresh_residual_t<7>(a, pb, pe, act);
    case 7: return refresh_residual_t<8>(a, pb, pe, act);
    default: return refresh_residual_t<9>(a, pb, pe, act);
  }
}

// act, m: the active list left by refresh_residual in this CTA, or nullptr
template <bool MIXED>
__device__ void refresh_correct_m(const SweepArgs& a, int pb, int pe, const int* act, int m) {
  switch (a.n_o) {
    case 1: refresh_correct_t<2, MIXED>(a, pb, pe, act, m); break;
    case 2: refresh_correct_t<3, MIXED>(a, pb, pe, act, m); break;
    case 3: refresh_correct_t<4, MIXED>(a, pb, pe, act, m); break;
    case 4: refresh_correct_t<5, MIXED>(a, pb, pe, act, m); break;
    case 5: refresh_correct_t<6, MIXED>(a, pb, pe, act, m); break;
    case 6: refresh_correct_t<7, MIXED>(a, pb, pe, act, m); break;
    case 7: refresh_correct_t<8, MIXED>(a, pb, pe, act, m); break;
    default: refresh_correct_t<9, MIXED>(a, pb, pe, act, m); break;
  }
}
__device__ void refresh_correct(const SweepArgs& a, int pb, int pe, const int* act = nullptr, int m = 0) {
  if (a.mixed) refresh_correct_m<true>(a, pb, pe, act, m);
  else refresh_correct_m<false>(a, pb, pe, act, m);
}

// ---------------------------------------------------------------- refresh correction, strips
// y = W x2 for the own rows (W symmetric, upper triangle current, x2 = v.r):
// the upper part sum_{i>=j} W[j][i] x2_i streams the own rows (one warp per
// row, four-wide reads), the lower part sum_{i<j} W[i][j] x2_i streams the
// rows above the own column strip, only those with b_i = 1 (x2 vanishes
// elsewhere).  x2 is staged in shared memory (all of it when it fits, else
// chunk by chunk) so that the inner loops read nothing but W from memory.
constexpr int CS_UNROLL = 16;  // lower part: rows in flight per warp

// bytes of dynamic shared memory of the running launch
__device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned b;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(b));
  return b;
}

// least shared memory the strips need (one 128-column chunk, 128 rows)
__host__ __device__ constexpr size_t cs_min_smem_bytes(int nv) {
  return (size_t)(kThreads / 32) * 32 * nv * sizeof(float2) + (size_t)nv * 128 * sizeof(float2) +
         128 * (sizeof(int) + nv * sizeof(float2));
}

// act: the ascending active-pixel list in global memory (or nullptr: every
// row), t_end: the number of its entries below pe - 1; smem: smem_bytes of
// shared memory
template <int NV, bool MIXED>
__device__ __noinline__ void correct_strips_t(const SweepArgs& a, int pb, int pe, const int* act, int t_end,
                                              float* smem, int smem_bytes) {
  const int n = a.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  float2* red = reinterpret_cast<float2*>(smem);  // [warps][NV][32]
  float2* xs = red + nw * NV * 32;                 // staged x2
  const int avail = smem_bytes - nw * NV * 32 * (int)sizeof(float2);
  // ---- upper part: rows g0 + warp of each group of nw own rows; chunks of cw columns
  const int n128 = (n + 127) & ~127;
  const int cw = min(n128, avail / (NV * (int)sizeof(float2)) / 128 * 128);
  const bool whole = cw >= n128;  // x2 staged once for every row group
  for (int g0 = pb; g0 < pe; g0 += nw) {
    const int j = g0 + warp;
    f2c acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = f2c{0.f, 0.f};
    const int cstart = whole ? 0 : (g0 & ~127);
    for (int c0 = cstart; c0 < n; c0 += cw) {
      if (!whole || g0 == pb) {
        __syncthreads();
        // column cc of the chunk at (cc & 3) * (cw / 4) + (cc >> 2): lanes read consecutive words
        for (int e = tid; e < NV * cw; e += blockDim.x) {
          const int q = e / cw, cc = e - q * cw, c = c0 + cc;
          xs[q * cw + (cc & 3) * (cw >> 2) + (cc >> 2)] = c < n ? x2f(a, q)[c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
      }
      if (j < pe) {
        const int kb = max(0, ((j & ~3) - c0) >> 7), ke = min(cw, n - c0 + 127) >> 7;
        for (int k0 = kb; k0 < ke; k0 += 8) {  // eight four-wide reads in flight per lane
          f2c w[8][4];
#pragma unroll
          for (int u8 = 0; u8 < 8; ++u8) {
            const int col = c0 + 128 * (k0 + u8) + 4 * lane;
            if (k0 + u8 < ke && col + 3 >= j && col < n) {
              w_row4<MIXED>(a, j, col, w[u8]);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) w[u8][u] = f2c{0.f, 0.f};
            }
          }
#pragma unroll
          for (int u8 = 0; u8 < 8; ++u8) {
            const int k = k0 + u8;
            if (k < ke) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int i = c0 + 128 * k + 4 * lane + u;
                if (i >= j && i < n) {
#pragma unroll
                  for (int q = 0; q < NV; ++q) {
                    const float2 x = xs[q * cw + u * (cw >> 2) + 32 * k + lane];
                    acc[q] = f2fma(w[u8][u], f2c{x.x, x.y}, acc[q]);
                  }
                }
              }
            }
          }
        }
      }
    }
    if (j < pe) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const f2c sum = f2sum(acc[q]);
        if (lane == 0) rvec(a, 3, q)[j] = mk(sum.x, sum.y);
      }
    }
  }
  // ---- lower part: own columns in blocks of 32 (lane = column), active rows i < pe - 1
  const int rcap = min(max(t_end, 1), avail / (int)(sizeof(int) + NV * sizeof(float2)));
  int* rows = reinterpret_cast<int*>(xs + NV * rcap);
  for (int cb = pb; cb < pe; cb += 32) {
    const int j = cb + lane;
    const bool colok = j < pe;
    f2c acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = f2c{0.f, 0.f};
    for (int t0 = 0; t0 < t_end; t0 += rcap) {
      const int cnt = min(rcap, t_end - t0);
      if (cb == pb || cnt < t_end) {  // staged once when every row fits
        __syncthreads();
        for (int e = tid; e < cnt; e += blockDim.x) rows[e] = act ? act[t0 + e] : t0 + e;
        __syncthreads();
        for (int e = tid; e < NV * cnt; e += blockDim.x) {
          const int q = e / cnt, tt = e - q * cnt;
          xs[q * rcap + tt] = x2f(a, q)[rows[tt]];
        }
        __syncthreads();
      }
      for (int tt = warp; tt < cnt; tt += CS_UNROLL * nw) {
        f2c w[CS_UNROLL];
#pragma unroll
        for (int u = 0; u < CS_UNROLL; ++u) {
          const int t2 = tt + u * nw;
          w[u] = f2c{0.f, 0.f};
          if (t2 < cnt) {
            const int i = rows[t2];
            if (colok && i < j) w[u] = w_upper<MIXED>(a, i, j);
          }
        }
#pragma unroll
        for (int u = 0; u < CS_UNROLL; ++u) {
          const int t2 = tt + u * nw;
          if (t2 < cnt) {
#pragma unroll
            for (int q = 0; q < NV; ++q) {
              const float2 x = xs[q * rcap + t2];
              acc[q] = f2fma(w[u], f2c{x.x, x.y}, acc[q]);
            }
          }
        }
      }
    }
    // sum the warps' column partials, then e, T += r + upper + lower
#pragma unroll
    for (int q = 0; q < NV; ++q) red[(warp * NV + q) * 32 + lane] = make_float2(acc[q].x, acc[q].y);
    __syncthreads();
    if (warp < NV && colok) {
      const int q = warp;
      float sx = 0.f, sy = 0.f;
      for (int w2 = 0; w2 < nw; ++w2) {
        sx += red[(w2 * NV + q) * 32 + lane].x;
        sy += red[(w2 * NV + q) * 32 + lane].y;
      }
      const c128 d = cadd(rvec(a, 0, q)[j], cadd(rvec(a, 3, q)[j], mk((double)sx, (double)sy)));
      c128* dst = q == 0 ? a.e + j : a.T + (size_t)(q - 1) * a.ldt + j;
      *dst = cadd(*dst, d);
    }
    __syncthreads();
  }
}

template <bool MIXED>
__device__ void correct_strips(const SweepArgs& a, int pb, int pe, const int* act, int t_end, float* smem,
                               int smem_bytes) {
  switch (a.n_o) {
    case 1: correct_strips_t<2, MIXED>(a, pb, pe, act, t_end, smem, smem_bytes); break;
    case 2: correct_strips_t<3, MIXED>(a, pb, pe, act, t_end, smem, smem_bytes); break;
    case 3: correct_strips_t<4, MIXED>(a, pb, pe, act, t_end, smem, smem_bytes); break;
    case 4: correct_strips_t<5, MIXED>(a, pb, pe, act, t_end, smem, smem_bytes); break;
    case 5: correct_strips_t<6, MIXED>(a, pb, pe, act, t_end, smem, smem_bytes); break;
    case 6: correct_strips_t<7, MIXED>(a, pb, pe, act, t_end, smem, smem_bytes); break;
    case 7: correct_strips_t<8, MIXED>(a, pb, pe, act, t_end, smem, smem_bytes); break;
    default: correct_strips_t<9, MIXED>(a, pb, pe, act, t_end, smem, smem_bytes); break;
  }
}

// partial o sums of pixels [pb, pe) -> opart[cta]
__device__ __noinline__ void ports_partial(const SweepArgs& a, int pb, int pe) {
  __shared__ c128 red[kMaxPorts][kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int p = 0; p < a.n_o; ++p) {
    c128 acc = mk(0.0, 0.0);
    for (int j = pb + threadIdx.x; j < pe; j += blockDim.x)
      acc = cfma(a.God[(size_t)p * a.n + j], cmul(a.v[j], a.e[j]), acc);
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) red[p][w] = acc;
  }
  __syncthreads();
  if (threadIdx.x < a.n_o) {
    c128 s = mk(0.0, 0.0);
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s = cadd(s, red[threadIdx.x][q]);
    a.opart[(size_t)blockIdx.x * a.n_o + threadIdx.x] = s;
  }
}

// o_p = c_o,p + sum over the CTAs of their partial sums (after a grid
// barrier): warp p adds port p's partials in a fixed lane order and tree, so
// every CTA obtains the same value; the FP64 adds run on one warp per port.
__device__ void ports_total(const SweepArgs& a, c128* o_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < a.n_o) {
    const int p = warp;
    c128 acc = mk(0.0, 0.0);
    for (int q = lane; q < (int)gridDim.x; q += 32) acc = cadd(acc, a.opart[(size_t)q * a.n_o + p]);
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) o_out[p] = cadd(a.co[p], acc);
  }
  __syncthreads();
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
  a.Gs = at<double>(c, L.gsum);
  a.God = c->God;
  a.cd = c->cd;
  a.co = c->co;
  a.op = c->obj;
  a.mixed = c->cfg.precision == PNGF_MIXED;
  a.ldl = L.ldl;
  a.R = L.R;
  a.Wr = at<float>(c, L.Wlo_re);
  a.Wi = at<float>(c, L.Wlo_im);
  a.X = at<float2>(c, L.X);
  a.xa = at<c128>(c, L.xa);
  a.rec = c->ws + L.rec;
  a.slots = at<unsigned long long>(c, L.slots);
  a.actg = at<int>(c, L.actg);
  a.G2 = a.mixed ? at<float4>(c, L.gsplit) : nullptr;
  a.xs = a.mixed ? at<float4>(c, L.xs) : nullptr;
  a.xadd = a.mixed ? at<float4>(c, L.xadd) : nullptr;
  a.tensor_fold = c->cfg.precision == PNGF_MIXED && c->cfg.tensor_fold;
  a.tcimgA = reinterpret_cast<unsigned char*>(c->ws) + L.tcimg;
  a.tcimgB = a.tcimgA + L.tcimgA_bytes;
  return a;
}


}  // namespace
}  // namespace pngf
