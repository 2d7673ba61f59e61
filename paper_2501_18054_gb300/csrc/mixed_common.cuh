// Device helpers of the mixed-precision path (FP32 maintained inverse plus an
// FP32 delayed rank-r set), shared by the persistent single-run kernel and
// the batched kernel.  Internal linkage; included after sweep_common.cuh.
#pragma once

#include "sweep_common.cuh"

namespace pngf {
namespace {

static_assert(sizeof(CandRecord) <= kRecordBytes, "candidate record slot");
constexpr int kMaxDelay = 128;

__device__ __forceinline__ CandRecord* rec_at(const SweepArgs& a, int slot, int q) {
  return reinterpret_cast<CandRecord*>(a.rec) + (size_t)slot * gridDim.x + q;
}

__device__ __forceinline__ void fill_record(const SweepArgs& a, CandRecord* r, int j, long long key,
                                            double gain, c128 alpha, c128 coef) {
  r->key = key;
  r->gain = gain;
  r->pixel = j;
  r->b = a.b[j];
  r->alpha = alpha;
  r->coef = coef;
  r->dv = a.dv[j];
  for (int p = 0; p < a.n_o; ++p) r->T[p] = a.T[(size_t)p * a.ldt + j];
}

// record of pixel j built from the state alone (single-call accept path)
__device__ __forceinline__ void fill_record_from_state(const SweepArgs& a, CandRecord* r, int j) {
  c128 dvj = a.dv[j];
  c128 delta = a.b[j] ? mk(-dvj.x, -dvj.y) : dvj;
  c128 dj = csub(mk(1.0, 0.0), cmul(delta, a.diag[j]));
  c128 alpha = cdiv(delta, dj);
  fill_record(a, r, j, 0, 0.0, alpha, cmul(alpha, a.e[j]));
}

__device__ __forceinline__ void pivot_from_record(const CandRecord& r, int n_o, Pivot& pv) {
  pv.k = r.pixel;
  pv.alpha = r.alpha;
  pv.coef = r.coef;
  for (int p = 0; p < n_o; ++p) pv.Tk[p] = r.T[p];
}

// W_lo(i, j) of the symmetric matrix through its upper triangle, promoted to FP64
__device__ __forceinline__ c128 wlo_sym(const SweepArgs& a, int i, int j) {
  int r = min(i, j), c = max(i, j);
  size_t o = (size_t)r * a.ldl + c;
  return mk((double)a.Wr[o], (double)a.Wi[o]);
}

// column assembly + state update for own pixels; appends c to the delayed set.
// One warp per pixel: lanes split the delayed sum, a shuffle reduction adds it.
__device__ void mixed_accept_own(const SweepArgs& a, const Pivot& pv, const float2* beta, int r, int pb, int pe) {
  constexpr int kChunk = 256;
  __shared__ c128 s_w[kChunk];
  __shared__ float2 s_sum[kChunk];
  const int g = threadIdx.x >> 4, gl = threadIdx.x & 15, ng = blockDim.x >> 4;
  const unsigned half = 0xffffu << (threadIdx.x & 16);
  for (int base = pb; base < pe; base += kChunk) {
    const int cnt = min(kChunk, pe - base);
    // U1: one thread per pixel fetches W_lo(k, j) (row k or column k)
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) s_w[t] = wlo_sym(a, pv.k, base + t);
    // U2: a 16-lane group per pixel forms the delayed sum in FP32
    for (int t = g; t < cnt; t += ng) {
      const float2* xj = a.X + (size_t)(base + t) * a.R;
      float px = 0.f, py = 0.f;
      for (int i = gl; i < r; i += 16) {
        float2 b = beta[i], x = xj[i];
        px = fmaf(b.x, x.x, fmaf(-b.y, x.y, px));
        py = fmaf(b.x, x.y, fmaf(b.y, x.x, py));
      }
      for (int off = 8; off > 0; off >>= 1) {
        px += __shfl_xor_sync(half, px, off);
        py += __shfl_xor_sync(half, py, off);
      }
      if (gl == 0) s_sum[t] = make_float2(px, py);
    }
    __syncthreads();
    // U3: one thread per pixel appends c_j and updates diag(W), e, T in FP64
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int j = base + t;
      c128 dj = a.diag[j], ej = a.e[j];
      c128 cj = mk(s_w[t].x + (double)s_sum[t].x, s_w[t].y + (double)s_sum[t].y);
      c128 aj = cmul(pv.alpha, cj);
      a.X[(size_t)j * a.R + r] = make_float2((float)cj.x, (float)cj.y);
      a.diag[j] = cfma(aj, cj, dj);
      a.e[j] = cfma(pv.coef, cj, ej);
#pragma unroll 1
      for (int p = 0; p < a.n_o; ++p) {
        c128* tp = a.T + (size_t)p * a.ldt + j;
        *tp = cfma(aj, pv.Tk[p], *tp);
      }
      if (j == pv.k) {
        uint8_t nb = a.b[j] ^ 1;
        a.b[j] = nb;
        a.v[j] = nb ? a.dv[j] : mk(0.0, 0.0);
      }
    }
    __syncthreads();
  }
}

// beta_i = alpha_i x_i[k] in FP32 for the delayed columns
__device__ __forceinline__ void make_beta(const SweepArgs& a, int k, int r, float2* beta) {
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    c128 al = a.xa[i];
    float2 x = a.X[(size_t)k * a.R + i];
    float ax = (float)al.x, ay = (float)al.y;
    beta[i] = make_float2(fmaf(ax, x.x, -ay * x.y), fmaf(ax, x.y, ay * x.x));
  }
}

// ---------------------------------------------------------------- flush
// W_lo[I, J] += sum_{i<r} alpha_i x_i[I] x_i[J]^T over the upper triangle of
// 64 x 64 tiles (diagonal tiles entirely).  FP32 operands in shared memory,
// FP32 accumulation, added into the FP32 planes.
constexpr int FT = 64;

struct f2x {
  float x, y;
};

// thread (ty, tx) owns rows ty + (FT/RU) u, u < RU, and columns tx + 16 v, v < 4
// of the 64 x 64 tile (RU = 2 for 512 threads, 4 for 256)
template <int RU>
__device__ __forceinline__ void flush_tile_fma(const SweepArgs& a, int r, const f2x* Ys, const f2x* Xs, int i0,
                                               int j0, int tx, int ty) {
  constexpr int LD = FT + 1;
  constexpr int RS = FT / RU;  // row stride between a thread's rows
  float accr[RU][4], acci[RU][4];
#pragma unroll
  for (int u = 0; u < RU; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) accr[u][v] = acci[u][v] = 0.f;
  for (int q = 0; q < r; ++q) {
    f2x y[RU], x[4];
#pragma unroll
    for (int u = 0; u < RU; ++u) y[u] = Ys[q * LD + ty + RS * u];
#pragma unroll
    for (int v = 0; v < 4; ++v) x[v] = Xs[q * LD + tx + 16 * v];
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        accr[u][v] = fmaf(y[u].x, x[v].x, fmaf(-y[u].y, x[v].y, accr[u][v]));
        acci[u][v] = fmaf(y[u].x, x[v].y, fmaf(y[u].y, x[v].x, acci[u][v]));
      }
  }
  const int n = a.n;
#pragma unroll
  for (int u = 0; u < RU; ++u) {
    int gi = i0 + ty + RS * u;
    if (gi >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int gj = j0 + tx + 16 * v;
      if (gj >= n) continue;
      size_t o = (size_t)gi * a.ldl + gj;
      a.Wr[o] += accr[u][v];
      a.Wi[o] += acci[u][v];
    }
  }
}

__device__ __noinline__ void flush_tiles(const SweepArgs& a, int r, float* smem, long long t_begin, long long t_step) {
  const int n = a.n;
  const int tn = (n + FT - 1) / FT;
  const long long n_tiles = (long long)tn * (tn + 1) / 2;
  constexpr int LD = FT + 1;                         // padded rows: no bank conflicts on the fills
  f2x* Ys = reinterpret_cast<f2x*>(smem);          // [r][LD]   rows of tile I, times alpha
  f2x* Xs = Ys + LD * kMaxDelay;                     // [r][LD]   rows of tile J
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x (blockDim / 16) threads
  __shared__ float2 s_alpha[kMaxDelay];
  __syncthreads();
  for (int q = threadIdx.x; q < r; q += blockDim.x) {
    c128 al = a.xa[q];
    s_alpha[q] = make_float2((float)al.x, (float)al.y);
  }
  for (long long t = t_begin; t < n_tiles; t += t_step) {
    int I, J;
    tri_rc(t, tn, I, J);
    const int i0 = I * FT, j0 = J * FT;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int rr = warp; rr < FT; rr += nw)
    for (int q = lane; q < r; q += 32) {
      int gi = i0 + rr, gj = j0 + rr;
      float2 al = s_alpha[q];
      float2 xi = gi < n ? a.X[(size_t)gi * a.R + q] : make_float2(0.f, 0.f);
      float2 xj = gj < n ? a.X[(size_t)gj * a.R + q] : make_float2(0.f, 0.f);
      Ys[q * LD + rr] = f2x{fmaf(al.x, xi.x, -al.y * xi.y), fmaf(al.x, xi.y, al.y * xi.x)};
      Xs[q * LD + rr] = f2x{xj.x, xj.y};
    }
    __syncthreads();
    if (blockDim.x >= 512)
      flush_tile_fma<2>(a, r, Ys, Xs, i0, j0, tx, ty);
    else
      flush_tile_fma<4>(a, r, Ys, Xs, i0, j0, tx, ty);
  }
}

constexpr size_t kFlushSmem = 2 * (FT + 1) * kMaxDelay * sizeof(f2x);

}  // namespace
}  // namespace pngf
