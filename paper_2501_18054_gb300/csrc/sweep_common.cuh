// Device building blocks shared by the FP64 and mixed-precision DBS kernels
// (scoring, selection, pivot, state update, grid barrier, FP64 refresh).
// Included by sweep.cu and sweep_mixed.cu; everything has internal linkage.
#pragma once

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
  float2* cpart;              // tile partial sums of the refresh correction
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
    const unsigned old = atomicAdd(&ctl->bar_count, 1u);
    const unsigned target = (old / P + 1) * P;
    unsigned long long it = 0;
    while ((int)(ld_volatile(&ctl->bar_count) - target) < 0) {
      if (++it > kSpinLimit) {
        latch_status(ctl, PNGF_ETIMEOUT);
        ok = 0;
        break;
      }
      if (it > 32) __nanosleep(32);
    }
    fence_acq_rel_gpu();  // acquire: every CTA's writes before the others' arrivals
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
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

// R0: x = v.[e, T] for own pixels
__device__ void refresh_x(const SweepArgs& a, int pb, int pe) {
  for (int j = pb + threadIdx.x; j < pe; j += blockDim.x) {
    c128 vj = a.v[j];
    rvec(a, 1, 0)[j] = cmul(vj, a.e[j]);
    for (int p = 0; p < a.n_o; ++p) rvec(a, 1, 1 + p)[j] = cmul(vj, a.T[(size_t)p * a.ldt + j]);
  }
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

// R1: residuals of own rows (row j of G dotted with x), and x2 = v.r.  With
// act (shared memory, room for n entries) only the columns of G at pixels
// with b_i = 1 are visited: x vanishes elsewhere, so the FP64 work follows the
// number of "on" pixels instead of n.
template <int NV>
__device__ __noinline__ int refresh_residual_t(const SweepArgs& a, int pb, int pe, int* act) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int m = act ? active_list(a, act) : a.n;
  for (int j = pb + warp; j < pe; j += nw) {
    const c128* g = a.G + (size_t)j * a.n;
    c128 acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = mk(0.0, 0.0);
    if (act) {
#pragma unroll 4
      for (int t = lane; t < m; t += 32) {
        const int i = act[t];
        c128 gi = g[i];
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] = cfma(gi, rvec(a, 1, q)[i], acc[q]);
      }
    } else {
#pragma unroll 4
      for (int i = lane; i < a.n; i += 32) {
        c128 gi = g[i];
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] = cfma(gi, rvec(a, 1, q)[i], acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      c128 sum = warp_sum(acc[q]);
      if (lane == 0) {
        c128 rhs = q == 0 ? a.cd[j] : a.God[(size_t)(q - 1) * a.n + j];
        c128 y = q == 0 ? a.e[j] : a.T[(size_t)(q - 1) * a.ldt + j];
        c128 r = cadd(csub(rhs, y), sum);
        rvec(a, 0, q)[j] = r;
        c128 x2 = cmul(a.v[j], r);
        x2f(a, q)[j] = make_float2((float)x2.x, (float)x2.y);
      }
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
__device__ __forceinline__ f2c w_upper(const SweepArgs& a, int i, int j) {
  if (a.mixed) {
    size_t o = (size_t)i * a.ldl + j;
    return f2c{a.Wr[o], a.Wi[o]};
  }
  return f2(a.W[(size_t)i * a.ldw + j]);
}

// four consecutive elements W(j, i0 .. i0+3) of the maintained W as FP32
// (i0 % 4 == 0; rows are padded to a multiple of 4 so the read stays inside
// the row; elements past n are masked by the caller)
__device__ __forceinline__ void w_row4(const SweepArgs& a, int j, int i0, f2c w[4]) {
  if (a.mixed) {
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
template <int NV>
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
      w_row4(a, j, i0, w);
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
template <int NV>
__device__ __noinline__ void refresh_correct_t(const SweepArgs& a, int pb, int pe, const int* act, int m) {
  __shared__ f2c red[kThreads / 32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  correct_upper<NV>(a, pb, pe);
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
        if (ii[u] >= 0 && colok && ii[u] < j) w[u] = w_upper(a, ii[u], j);
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
__device__ void refresh_correct(const SweepArgs& a, int pb, int pe, const int* act = nullptr, int m = 0) {
  switch (a.n_o) {
    case 1: refresh_correct_t<2>(a, pb, pe, act, m); break;
    case 2: refresh_correct_t<3>(a, pb, pe, act, m); break;
    case 3: refresh_correct_t<4>(a, pb, pe, act, m); break;
    case 4: refresh_correct_t<5>(a, pb, pe, act, m); break;
    case 5: refresh_correct_t<6>(a, pb, pe, act, m); break;
    case 6: refresh_correct_t<7>(a, pb, pe, act, m); break;
    case 7: refresh_correct_t<8>(a, pb, pe, act, m); break;
    default: refresh_correct_t<9>(a, pb, pe, act, m); break;
  }
}

// ---------------------------------------------------------------- refresh correction, tiled
// The persistent kernels form y = W x2 (x2 = v.r, W symmetric with its upper
// triangle current) by 64 x 64 tiles of the upper triangle: a tile (I, J),
// I <= J, is read once and yields both its row sums W[I, J] x2[J] (for block
// I) and its column sums W[I, J]^T x2[I] (for block J); on a diagonal tile the
// row sums take the upper part including the diagonal and the column sums
// the strict upper part.  Partial sums go to cpart, tile by tile, and the
// owner of a row adds them in a fixed order (deterministic, no atomics).
constexpr int CT = 64;

__host__ __device__ __forceinline__ long long ct_tiles(int n) {
  const long long tn = (n + CT - 1) / CT;
  return tn * (tn + 1) / 2;
}
__device__ __forceinline__ long long ct_index(int I, int J, int tn) {
  return (long long)I * tn - (long long)I * (I - 1) / 2 + (J - I);
}
// cpart[((t * 2 + side) * NV + q) * CT + i], side 0: row sums, 1: column sums
__device__ __forceinline__ float2* ct_part(const SweepArgs& a, long long t, int side, int q, int nv) {
  return a.cpart + (((size_t)t * 2 + side) * nv + q) * CT;
}
// shared memory of correct_tiles_t: x2 of both blocks and one column-sum stage
__host__ __device__ constexpr size_t ct_smem_bytes(int nv) {
  return (size_t)2 * nv * CT * sizeof(float2) + (size_t)(kThreads / 32) * CT * sizeof(float2);
}

template <int NV>
__device__ __noinline__ void correct_tiles_t(const SweepArgs& a, float* smem) {
  const int n = a.n, tn = (n + CT - 1) / CT;
  const long long T = ct_tiles(n);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tid & 15, ty = tid >> 4;  // columns 4 tx .. 4 tx + 3, rows 2 ty, 2 ty + 1
  float2* xJ = reinterpret_cast<float2*>(smem);  // [NV][CT]
  float2* xI = xJ + NV * CT;                     // [NV][CT]
  float2* cst = xI + NV * CT;                    // [warps][CT]
  for (long long t = blockIdx.x; t < T; t += gridDim.x) {
    int I, J;
    tri_rc(t, tn, I, J);
    const int i0 = I * CT, j0 = J * CT;
    const bool diag = I == J;
    __syncthreads();
    for (int q = tid; q < NV * CT; q += blockDim.x) {
      const int v = q / CT, c = q - v * CT;
      xJ[q] = j0 + c < n ? x2f(a, v)[j0 + c] : make_float2(0.f, 0.f);
      xI[q] = i0 + c < n ? x2f(a, v)[i0 + c] : make_float2(0.f, 0.f);
    }
    // the tile in registers (masked entries are zero)
    f2c w[2][4];
    const int cg = j0 + 4 * tx;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int rg = i0 + 2 * ty + u;
      if (rg < n && cg < n) {
        w_row4(a, rg, cg, w[u]);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) w[u][c] = f2c{0.f, 0.f};
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (cg + c >= n || (diag && cg + c < rg)) w[u][c] = f2c{0.f, 0.f};  // upper part only
    }
    __syncthreads();
#pragma unroll 1
    for (int q = 0; q < NV; ++q) {
      // row sums over this thread's four columns, then over the 16 column groups
      f2c rs[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        rs[u] = f2c{0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float2 x = xJ[q * CT + 4 * tx + c];
          rs[u] = f2fma(w[u][c], f2c{x.x, x.y}, rs[u]);
        }
#pragma unroll
        for (int off = 1; off < 16; off <<= 1) {
          rs[u].x += __shfl_xor_sync(0xffffffffu, rs[u].x, off);
          rs[u].y += __shfl_xor_sync(0xffffffffu, rs[u].y, off);
        }
      }
      if (tx == 0) {
        float2* pr = ct_part(a, t, 0, q, NV);
        pr[2 * ty] = make_float2(rs[0].x, rs[0].y);
        pr[2 * ty + 1] = make_float2(rs[1].x, rs[1].y);
      }
      // column sums over this thread's two rows (strict upper part on a diagonal tile)
      f2c cs[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        cs[c] = f2c{0.f, 0.f};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (diag && cg + c == i0 + 2 * ty + u) continue;  // the diagonal belongs to the row sums
          const float2 x = xI[q * CT + 2 * ty + u];
          cs[c] = f2fma(w[u][c], f2c{x.x, x.y}, cs[c]);
        }
        cs[c].x += __shfl_xor_sync(0xffffffffu, cs[c].x, 16);
        cs[c].y += __shfl_xor_sync(0xffffffffu, cs[c].y, 16);
      }
      if (lane < 16)
#pragma unroll
        for (int c = 0; c < 4; ++c) cst[warp * CT + 4 * tx + c] = make_float2(cs[c].x, cs[c].y);
      __syncthreads();
      if (tid < CT) {
        float sx = 0.f, sy = 0.f;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) {
          sx += cst[w2 * CT + tid].x;
          sy += cst[w2 * CT + tid].y;
        }
        ct_part(a, t, 1, q, NV)[tid] = make_float2(sx, sy);
      }
      __syncthreads();
    }
  }
}

// after a grid barrier: e, T of own rows += r + y, y summed from the tile
// partials in a fixed order (one warp per row, lanes over the tiles)
template <int NV>
__device__ __noinline__ void correct_finish_t(const SweepArgs& a, int pb, int pe) {
  const int n = a.n, tn = (n + CT - 1) / CT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = pb + warp; j < pe; j += nw) {
    const int B = j / CT, rho = j - B * CT;
    const int nterm = tn + 1;  // row sums of tiles (B, J >= B), column sums of tiles (I <= B, B)
    float sx[NV], sy[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) sx[q] = sy[q] = 0.f;
#pragma unroll 4
    for (int u = lane; u < nterm; u += 32) {
      const float2* base = u < tn - B ? ct_part(a, ct_index(B, B + u, tn), 0, 0, NV)
                                      : ct_part(a, ct_index(u - (tn - B), B, tn), 1, 0, NV);
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const float2 p = base[q * CT + rho];
        sx[q] += p.x;
        sy[q] += p.y;
      }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      for (int off = 16; off > 0; off >>= 1) {
        sx[q] += __shfl_xor_sync(0xffffffffu, sx[q], off);
        sy[q] += __shfl_xor_sync(0xffffffffu, sy[q], off);
      }
    }
    if (lane < NV) {  // lane q updates vector q (e for q = 0, row q - 1 of T otherwise)
      float fx = 0.f, fy = 0.f;
#pragma unroll
      for (int q = 0; q < NV; ++q)
        if (q == lane) {
          fx = sx[q];
          fy = sy[q];
        }
      const c128 d = cadd(rvec(a, 0, lane)[j], mk((double)fx, (double)fy));
      c128* dst = lane == 0 ? a.e + j : a.T + (size_t)(lane - 1) * a.ldt + j;
      *dst = cadd(*dst, d);
    }
  }
}

__device__ void correct_tiles(const SweepArgs& a, float* smem) {
  switch (a.n_o) {
    case 1: correct_tiles_t<2>(a, smem); break;
    case 2: correct_tiles_t<3>(a, smem); break;
    case 3: correct_tiles_t<4>(a, smem); break;
    case 4: correct_tiles_t<5>(a, smem); break;
    case 5: correct_tiles_t<6>(a, smem); break;
    case 6: correct_tiles_t<7>(a, smem); break;
    case 7: correct_tiles_t<8>(a, smem); break;
    default: correct_tiles_t<9>(a, smem); break;
  }
}

__device__ void correct_finish(const SweepArgs& a, int pb, int pe) {
  switch (a.n_o) {
    case 1: correct_finish_t<2>(a, pb, pe); break;
    case 2: correct_finish_t<3>(a, pb, pe); break;
    case 3: correct_finish_t<4>(a, pb, pe); break;
    case 4: correct_finish_t<5>(a, pb, pe); break;
    case 5: correct_finish_t<6>(a, pb, pe); break;
    case 6: correct_finish_t<7>(a, pb, pe); break;
    case 7: correct_finish_t<8>(a, pb, pe); break;
    default: correct_finish_t<9>(a, pb, pe); break;
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
  a.mixed = c->cfg.precision == PNGF_MIXED;
  a.ldl = L.ldl;
  a.R = L.R;
  a.Wr = at<float>(c, L.Wlo_re);
  a.Wi = at<float>(c, L.Wlo_im);
  a.X = at<float2>(c, L.X);
  a.xa = at<c128>(c, L.xa);
  a.rec = c->ws + L.rec;
  a.slots = at<unsigned long long>(c, L.slots);
  a.cpart = at<float2>(c, L.cpart);
  a.tensor_fold = c->cfg.precision == PNGF_MIXED && c->cfg.tensor_fold;
  a.tcimgA = reinterpret_cast<unsigned char*>(c->ws) + L.tcimg;
  a.tcimgB = a.tcimgA + L.tcimgA_bytes;
  return a;
}


}  // namespace
}  // namespace pngf
