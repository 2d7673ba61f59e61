// Initial factorisation of the reduced system and formation of the maintained
// state (the inverse of the paper's initial system matrix C_0, section
// "Direct binary search optimization"; field form of Supplementary Note 4):
//
//   M = I - G diag(v),  v = dv .* b
//   LU = P M            blocked right-looking LU with partial pivoting, FP64
//   [W | e] = M^-1 [G | c_d]   forward / backward substitution, blocked
//   T = G_od + (G_od diag(v)) W,  o = c_o + G_od (v .* e),  diag(W)
//
// Everything is complex128 and row-major.  The trailing updates are complex
// GEMMs on the FP64 pipe (four DFMA per complex multiply-add): on this GPU the
// FP64 rate is about 1.2 TFLOP/s, so every kernel here is FP64-pipe bound.
#include <cstdio>

#include "sweep_common.cuh"

namespace pngf {
namespace {

constexpr int NB = 32;  // panel width / block size of the substitutions
constexpr int kCoopPanelRows = 256;  // taller panels are factored by many CTAs

// ---------------------------------------------------------------- M = I - G V
__global__ void build_system(const c128* __restrict__ G, const c128* __restrict__ dv,
                             const uint8_t* __restrict__ b, int n, int ldw, c128* __restrict__ LU,
                             c128* __restrict__ v_out, uint8_t* __restrict__ b_out) {
  // one matrix row per blockIdx.y, columns over x
  int i = blockIdx.y;
  const c128* g = G + (size_t)i * n;
  c128* m = LU + (size_t)i * ldw;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    c128 vj = b[j] ? dv[j] : mk(0.0, 0.0);
    c128 gij = g[j];
    c128 mij = mk(-(gij.x * vj.x - gij.y * vj.y), -(gij.x * vj.y + gij.y * vj.x));
    if (j == i) mij.x += 1.0;
    m[j] = mij;
    if (i == 0) {
      v_out[j] = vj;
      b_out[j] = b[j] ? 1 : 0;
    }
  }
}

// ---------------------------------------------------------------- panel
// Factor rows [j0, n) x columns [j0, j0+jb) in place with partial pivoting.
// One CTA of 1024 threads; warp w handles rows j0 + w, j0 + w + 32, ...;
// lane l handles panel column j0 + l.  The magnitude |re| + |im| chooses the
// pivot (ties -> lowest row).
__global__ void __launch_bounds__(1024) panel_factor(c128* __restrict__ A, int n, int lda, int j0,
                                                     int jb, int* __restrict__ ipiv,
                                                     Control* __restrict__ ctl) {
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ c128 urow[NB];
  __shared__ int piv_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool active_lane = lane < jb;
  // running maximum of column (j0 + jj) over this warp's rows, kept by lane jj
  double best_v = -1.0;
  int best_i = 0x7fffffff;
  // initial pivot search on column j0: lane 0 of each warp scans its rows
  for (int r = j0 + warp; r < n; r += 32) {
    double a = cabs1(A[(size_t)r * lda + j0]);
    if (lane == 0 && (a > best_v)) { best_v = a; best_i = r; }
  }
  for (int jj = 0; jj < jb; ++jj) {
    const int col = j0 + jj;
    // ---- reduce the candidate held by lane jj of every warp
    double cv = __shfl_sync(0xffffffffu, best_v, jj);
    int ci = __shfl_sync(0xffffffffu, best_i, jj);
    if (lane == 0) { red_v[warp] = cv; red_i[warp] = ci; }
    __syncthreads();
    if (warp == 0) {
      double vv = red_v[lane];
      int ii = red_i[lane];
      for (int off = 16; off > 0; off >>= 1) {
        double ov = __shfl_down_sync(0xffffffffu, vv, off);
        int oi = __shfl_down_sync(0xffffffffu, ii, off);
        if (ov > vv || (ov == vv && oi < ii)) { vv = ov; ii = oi; }
      }
      if (lane == 0) {
        if (!(vv > 0.0)) {  // exact zero (or NaN) column: singular
          latch_status(ctl, PNGF_ESINGULAR);
          ii = col;
        }
        piv_s = ii;
        ipiv[col] = ii;
      }
    }
    __syncthreads();
    const int p = piv_s;
    // ---- swap rows col and p inside the panel
    if (p != col && threadIdx.x < jb) {
      c128 t = A[(size_t)col * lda + j0 + threadIdx.x];
      A[(size_t)col * lda + j0 + threadIdx.x] = A[(size_t)p * lda + j0 + threadIdx.x];
      A[(size_t)p * lda + j0 + threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x < jb) urow[threadIdx.x] = A[(size_t)col * lda + j0 + threadIdx.x];
    __syncthreads();
    const c128 piv = urow[jj];
    const c128 inv = cdiv(mk(1.0, 0.0), piv);
    // ---- scale column col below the diagonal and update the trailing panel columns;
    //      track the next column's maximum on lane jj+1
    best_v = -1.0;
    best_i = 0x7fffffff;
    const c128 u = active_lane ? urow[lane] : mk(0.0, 0.0);
    for (int r = col + 1 + warp; r < n; r += 32) {
      c128* row = A + (size_t)r * lda + j0;
      c128 a = active_lane ? row[lane] : mk(0.0, 0.0);
      double lx = __shfl_sync(0xffffffffu, a.x, jj);
      double ly = __shfl_sync(0xffffffffu, a.y, jj);
      c128 lr = cmul(mk(lx, ly), inv);
      if (lane == jj) {
        row[lane] = lr;
      } else if (active_lane && lane > jj) {
        c128 na = cfms(lr, u, a);
        row[lane] = na;
        if (lane == jj + 1) {
          double m = cabs1(na);
          if (m > best_v) { best_v = m; best_i = r; }
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- panel, many CTAs
// The same factorisation of rows [j0, n) x columns [j0, j0+jb) spread over a
// cooperative grid: CTA q owns a contiguous chunk of the rows.  Per column:
// every CTA reduces the CTAs' candidates (same fixed order everywhere: the
// same pivot), the owners of the pivot row and of the diagonal row stage
// them, a grid barrier, the swap and the update of every CTA's own rows
// (tracking the next column's candidate), a grid barrier.  The FP64 work of a
// panel is spread over the SMs instead of one, where a single CTA is held to
// one SM's share of the FP64 pipe.
constexpr int PC_THREADS = 256;

__device__ __forceinline__ void pc_better(double& v, long long& i, double ov, long long oi) {
  if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
}

__global__ void __launch_bounds__(PC_THREADS) panel_factor_coop(c128* __restrict__ A, int n, int lda, int j0, int jb,
                                                                int* __restrict__ ipiv, Control* __restrict__ ctl,
                                                                double* __restrict__ pv, long long* __restrict__ pi,
                                                                c128* __restrict__ rowbuf) {
  __shared__ double red_v[PC_THREADS / 32];
  __shared__ long long red_i[PC_THREADS / 32];
  __shared__ c128 urow[NB];
  __shared__ int piv_s;
  const int P = gridDim.x, cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rows = n - j0;
  const int rb = j0 + (int)((long long)rows * cta / P), re = j0 + (int)((long long)rows * (cta + 1) / P);
  const bool active_lane = lane < jb;
  // this CTA's candidate for column j0
  {
    double v = -1.0;
    long long idx = LLONG_MAX;
    for (int r = rb + tid; r < re; r += blockDim.x) pc_better(v, idx, cabs1(A[(size_t)r * lda + j0]), r);
    for (int off = 16; off > 0; off >>= 1)
      pc_better(v, idx, __shfl_xor_sync(0xffffffffu, v, off), __shfl_xor_sync(0xffffffffu, idx, off));
    if (lane == 0) { red_v[warp] = v; red_i[warp] = idx; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < PC_THREADS / 32; ++w) pc_better(v, idx, red_v[w], red_i[w]);
      pv[cta] = v;
      pi[cta] = idx;
    }
  }
  if (!grid_sync(ctl)) return;
  for (int jj = 0; jj < jb; ++jj) {
    const int col = j0 + jj, par = jj & 1;
    // ---- the pivot: every CTA reduces the P candidates in the same order
    double v = -1.0;
    long long idx = LLONG_MAX;
    for (int q = tid; q < P; q += blockDim.x) pc_better(v, idx, pv[par * P + q], pi[par * P + q]);
    for (int off = 16; off > 0; off >>= 1)
      pc_better(v, idx, __shfl_xor_sync(0xffffffffu, v, off), __shfl_xor_sync(0xffffffffu, idx, off));
    __syncthreads();
    if (lane == 0) { red_v[warp] = v; red_i[warp] = idx; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < PC_THREADS / 32; ++w) pc_better(v, idx, red_v[w], red_i[w]);
      int p = (int)idx;
      if (!(v > 0.0)) {  // exact zero (or NaN) column: singular
        if (cta == 0) latch_status(ctl, PNGF_ESINGULAR);
        p = col;
      }
      piv_s = p;
      if (cta == 0) ipiv[col] = p;
    }
    __syncthreads();
    const int p = piv_s;
    // ---- stage the pivot row (slot 0) and the diagonal row (slot 1)
    if (p >= rb && p < re && tid < jb) rowbuf[tid] = A[(size_t)p * lda + j0 + tid];
    if (col >= rb && col < re && tid < jb) rowbuf[NB + tid] = A[(size_t)col * lda + j0 + tid];
    if (!grid_sync(ctl)) return;
    if (tid < jb) urow[tid] = rowbuf[tid];
    if (p != col) {
      if (col >= rb && col < re && tid < jb) A[(size_t)col * lda + j0 + tid] = rowbuf[tid];
      if (p >= rb && p < re && tid < jb) A[(size_t)p * lda + j0 + tid] = rowbuf[NB + tid];
    }
    __syncthreads();
    // ---- scale column col below the diagonal, update the trailing panel
    //      columns of the own rows, track the next column's candidate
    const c128 inv = cdiv(mk(1.0, 0.0), urow[jj]);
    const c128 u = active_lane ? urow[lane] : mk(0.0, 0.0);
    double bv = -1.0;
    long long bi = LLONG_MAX;
    for (int r = max(rb, col + 1) + warp; r < re; r += PC_THREADS / 32) {
      c128* row = A + (size_t)r * lda + j0;
      const c128 a = active_lane ? row[lane] : mk(0.0, 0.0);
      const double lx = __shfl_sync(0xffffffffu, a.x, jj);
      const double ly = __shfl_sync(0xffffffffu, a.y, jj);
      const c128 lr = cmul(mk(lx, ly), inv);
      if (lane == jj) {
        row[lane] = lr;
      } else if (active_lane && lane > jj) {
        const c128 na = cfms(lr, u, a);
        row[lane] = na;
        if (lane == jj + 1) pc_better(bv, bi, cabs1(na), r);
      }
    }
    if (jj + 1 < jb) {
      // lane jj + 1 of each warp holds the warp's candidate
      bv = __shfl_sync(0xffffffffu, bv, jj + 1);
      bi = __shfl_sync(0xffffffffu, bi, jj + 1);
      __syncthreads();
      if (lane == 0) { red_v[warp] = bv; red_i[warp] = bi; }
      __syncthreads();
      if (tid == 0) {
        for (int w = 1; w < PC_THREADS / 32; ++w) pc_better(bv, bi, red_v[w], red_i[w]);
        pv[(par ^ 1) * P + cta] = bv;
        pi[(par ^ 1) * P + cta] = bi;
      }
    }
    if (!grid_sync(ctl)) return;
  }
}

// ---------------------------------------------------------------- row swaps
// Apply the panel's interchanges (rows j0.. j0+jb-1 with ipiv[...]) to the
// columns outside the panel.
__global__ void apply_swaps(c128* __restrict__ A, int n, int lda, int j0, int jb,
                            const int* __restrict__ ipiv) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n || (c >= j0 && c < j0 + jb)) return;
  for (int jj = 0; jj < jb; ++jj) {
    int r = j0 + jj, p = ipiv[r];
    if (p != r) {
      c128 t = A[(size_t)r * lda + c];
      A[(size_t)r * lda + c] = A[(size_t)p * lda + c];
      A[(size_t)p * lda + c] = t;
    }
  }
}

// ---------------------------------------------------------------- triangular blocks
// B[0:jb, 0:ncols] = L^-1 B (L unit lower jb x jb) or U^-1 B (U upper, non-unit).
// One thread per right-hand-side column; the jb x jb block lives in shared memory.
template <bool kLower>
__global__ void __launch_bounds__(256) trsm_block(const c128* __restrict__ T, int ldt, int jb,
                                                  c128* __restrict__ B, int ldb, int ncols) {
  __shared__ c128 Ts[NB][NB + 1];
  __shared__ c128 dinv[NB];
  for (int idx = threadIdx.x; idx < jb * jb; idx += blockDim.x) {
    int i = idx / jb, j = idx % jb;
    Ts[i][j] = T[(size_t)i * ldt + j];
  }
  __syncthreads();
  if (!kLower && threadIdx.x < jb) dinv[threadIdx.x] = cdiv(mk(1.0, 0.0), Ts[threadIdx.x][threadIdx.x]);
  __syncthreads();
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  c128 x[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) x[i] = (i < jb) ? B[(size_t)i * ldb + c] : mk(0.0, 0.0);
  if (kLower) {
#pragma unroll
    for (int i = 1; i < NB; ++i) {
      if (i < jb) {
        c128 s = x[i];
#pragma unroll
        for (int l = 0; l < NB; ++l)
          if (l < i) s = cfms(Ts[i][l], x[l], s);
        x[i] = s;
      }
    }
  } else {
#pragma unroll
    for (int i = NB - 1; i >= 0; --i) {
      if (i < jb) {
        c128 s = x[i];
#pragma unroll
        for (int l = 0; l < NB; ++l)
          if (l > i && l < jb) s = cfms(Ts[i][l], x[l], s);
        x[i] = cmul(s, dinv[i]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < jb) B[(size_t)i * ldb + c] = x[i];
}

// ---------------------------------------------------------------- complex GEMM
// C[M x N] -= A[M x K] * B[K x N], row-major.  64 x 64 tile per CTA, 256
// threads, each owning a 4 x 4 block of complex outputs (rows ty + 16 r,
// columns tx + 16 c); K in chunks of 16 through shared memory.
constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

__global__ void __launch_bounds__(256) zgemm_sub(int M, int N, int K, const c128* __restrict__ A,
                                                 int lda, const c128* __restrict__ B, int ldb,
                                                 c128* __restrict__ C, int ldc) {
  __shared__ c128 As[GB_K][GB_M];
  __shared__ c128 Bs[GB_K][GB_N];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
  c128 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = mk(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += GB_K) {
    // A tile: 64 rows x 16 k -> As[k][m]
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = threadIdx.x + q * 256;
      int mm = idx >> 4, kk = idx & 15;
      int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : mk(0.0, 0.0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int idx = threadIdx.x + q * 256;
      int kk = idx >> 6, nn = idx & 63;
      int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < K && gn < N) ? B[(size_t)gk * ldb + gn] : mk(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      c128 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = cfma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int gm = m0 + ty + 16 * r;
    if (gm >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int gn = n0 + tx + 16 * c;
      if (gn < N) {
        c128* p = C + (size_t)gm * ldc + gn;
        *p = csub(*p, acc[r][c]);
      }
    }
  }
}

void gemm_sub(cudaStream_t s, int M, int N, int K, const c128* A, int lda, const c128* B, int ldb,
              c128* C, int ldc) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  dim3 grid((N + GB_N - 1) / GB_N, (M + GB_M - 1) / GB_M);
  zgemm_sub<<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
}

// ---------------------------------------------------------------- permutation of the RHS
__global__ void pivots_to_perm(const int* __restrict__ ipiv, int n, int* __restrict__ perm) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int i = 0; i < n; ++i) {
    int p = ipiv[i];
    int t = perm[i];
    perm[i] = perm[p];
    perm[p] = t;
  }
}

// Right-hand side of the substitutions: W[i][0:n] = G[perm[i]][:], W[i][n] = c_d[perm[i]]
__global__ void gather_rhs(const c128* __restrict__ G, const c128* __restrict__ cd, int n,
                           const int* __restrict__ perm, c128* __restrict__ W, int ldw) {
  int i = blockIdx.y;
  int pi = perm[i];
  const c128* s = G + (size_t)pi * n;
  c128* d = W + (size_t)i * ldw;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += gridDim.x * blockDim.x)
    d[j] = (j < n) ? s[j] : cd[pi];
}

// ---------------------------------------------------------------- state formation
// T[p][j] = G_od[p][j] + sum_i (G_od[p][i] v_i) W[i][j]; one thread per column j.
__global__ void __launch_bounds__(256) form_T(const c128* __restrict__ W, int n, int ldw,
                                              const c128* __restrict__ God, const c128* __restrict__ v,
                                              int n_o, c128* __restrict__ T, int ldt) {
  __shared__ c128 gv[kMaxPorts][64];
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  c128 acc[kMaxPorts];
  for (int p = 0; p < kMaxPorts; ++p) acc[p] = mk(0.0, 0.0);
  for (int i0 = 0; i0 < n; i0 += 64) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < n_o * 64; idx += blockDim.x) {
      int p = idx / 64, ii = idx % 64, i = i0 + ii;
      gv[p][ii] = (i < n) ? cmul(God[(size_t)p * n + i], v[i]) : mk(0.0, 0.0);
    }
    __syncthreads();
    if (j < n) {
      int iend = min(64, n - i0);
      for (int ii = 0; ii < iend; ++ii) {
        c128 w = W[(size_t)(i0 + ii) * ldw + j];
        FOR_PORTS(p, n_o) acc[p] = cfma(gv[p][ii], w, acc[p]);
      }
    }
  }
  if (j < n)
    FOR_PORTS(p, n_o) T[(size_t)p * ldt + j] = cadd(God[(size_t)p * n + j], acc[p]);
}

// diag(W), e = column n of the solved RHS
__global__ void extract_diag_e(const c128* __restrict__ W, int n, int ldw, c128* __restrict__ diag,
                               c128* __restrict__ e) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    diag[j] = W[(size_t)j * ldw + j];
    e[j] = W[(size_t)j * ldw + n];
  }
}

// o = c_o + G_od (v .* e), objective, reset of the sweep counters.  One CTA.
__global__ void __launch_bounds__(256) form_o(const c128* __restrict__ God, const c128* __restrict__ co,
                                              const c128* __restrict__ v, const c128* __restrict__ e,
                                              int n, ObjParams op, Control* __restrict__ ctl) {
  __shared__ c128 red[kMaxPorts][256];
  c128 acc[kMaxPorts];
  for (int p = 0; p < kMaxPorts; ++p) acc[p] = mk(0.0, 0.0);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    c128 ve = cmul(v[j], e[j]);
    FOR_PORTS(p, op.n_o) acc[p] = cfma(God[(size_t)p * n + j], ve, acc[p]);
  }
  FOR_PORTS(p, op.n_o) red[p][threadIdx.x] = acc[p];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      FOR_PORTS(p, op.n_o) red[p][threadIdx.x] = cadd(red[p][threadIdx.x], red[p][threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    c128 o[kMaxPorts];
    FOR_PORTS(p, op.n_o) {
      o[p] = cadd(co[p], red[p][0]);
      ctl->o[p] = o[p];
    }
    ctl->f = objective_of(op, o);
    ctl->factored = 1;
    ctl->n_acc_total = 0;
    ctl->since_refresh = 0;
    ctl->r_delay = 0;
  }
}

// S = Re G + Im G (n x n, row-major), the third real matrix of the refresh's
// three-multiplication complex products
__global__ void gsum_kernel(const c128* __restrict__ G, long long nn, double* __restrict__ S) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const c128 g = G[i];
    S[i] = g.x + g.y;
  }
}

// G as unevaluated sums of two FP32 values per real part, hi = fl32(g) and
// lo = fl32(g - hi) (48 significant bits), for the double-float refresh
// residual of the mixed search: (Re hi, Im hi, Re lo, Im lo), so that the
// (Re, Im) pairs of the hi and of the lo parts are 64-bit operands
__global__ void gsplit_kernel(const c128* __restrict__ G, long long nn, float4* __restrict__ G2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const c128 g = G[i];
    const float rh = (float)g.x, ih = (float)g.y;
    G2[i] = make_float4(rh, ih, (float)(g.x - (double)rh), (float)(g.y - (double)ih));
  }
}

}  // namespace

// ---------------------------------------------------------------- driver
pngf_status factor_fp64(pngf_ctx* c, const uint8_t* b) {
  const int n = c->cfg.n_d, n_o = c->cfg.n_o;
  const int ldw = c->L.ldw;
  cudaStream_t s = c->stream;
  c128* LU = at<c128>(c, c->L.LU);
  c128* W = at<c128>(c, c->L.W);
  int* ipiv = at<int>(c, c->L.ipiv);
  int* perm = ipiv + n;
  Control* ctl = at<Control>(c, c->L.ctl);
  c128* v = at<c128>(c, c->L.v);
  uint8_t* bb = at<uint8_t>(c, c->L.b);
  c128* diag = at<c128>(c, c->L.diag);
  c128* e = at<c128>(c, c->L.e);
  c128* T = at<c128>(c, c->L.T);
  {
    dim3 grid((n + 255) / 256 > 8 ? 8 : (n + 255) / 256, n);
    build_system<<<grid, 256, 0, s>>>(c->G, c->dv, b, n, ldw, LU, v, bb);
  }
  gsum_kernel<<<c->n_sm * 4, 256, 0, s>>>(c->G, (long long)n * n, at<double>(c, c->L.gsum));
  if (c->cfg.precision == PNGF_MIXED)
    gsplit_kernel<<<c->n_sm * 4, 256, 0, s>>>(c->G, (long long)n * n, at<float4>(c, c->L.gsplit));
  // LU with partial pivoting
  for (int j0 = 0; j0 < n; j0 += NB) {
    int jb = n - j0 < NB ? n - j0 : NB;
    const int rows = n - j0;
    if (rows > kCoopPanelRows) {
      int P = (rows + 31) / 32;
      if (P > c->n_sm) P = c->n_sm;
      if (cudaMemsetAsync(&ctl->bar_count, 0, sizeof(unsigned), s) != cudaSuccess) return PNGF_ECUDA;
      double* pv = reinterpret_cast<double*>(c->ws + c->L.part + 2 * (size_t)c->L.n_part * sizeof(long long));
      long long* pi = reinterpret_cast<long long*>(c->ws + c->L.part);
      c128* rowbuf = at<c128>(c, c->L.rbuf);
      void* params[] = {&LU, (void*)&n, (void*)&ldw, &j0, &jb, &ipiv, &ctl, &pv, &pi, &rowbuf};
      if (cudaLaunchCooperativeKernel((const void*)panel_factor_coop, dim3(P), dim3(PC_THREADS), params, 0, s) !=
          cudaSuccess)
        return PNGF_ECUDA;
    } else {
      panel_factor<<<1, 1024, 0, s>>>(LU, n, ldw, j0, jb, ipiv, ctl);
    }
    apply_swaps<<<(n + 255) / 256, 256, 0, s>>>(LU, n, ldw, j0, jb, ipiv);
    int rest = n - j0 - jb;
    if (rest > 0) {
      trsm_block<true><<<(rest + 255) / 256, 256, 0, s>>>(LU + (size_t)j0 * ldw + j0, ldw, jb,
                                                           LU + (size_t)j0 * ldw + j0 + jb, ldw, rest);
      gemm_sub(s, rest, rest, jb, LU + (size_t)(j0 + jb) * ldw + j0, ldw,
               LU + (size_t)j0 * ldw + j0 + jb, ldw, LU + (size_t)(j0 + jb) * ldw + j0 + jb, ldw);
    }
  }
  // RHS permutation: W = P [G | c_d]
  pivots_to_perm<<<1, 1, 0, s>>>(ipiv, n, perm);
  {
    dim3 grid((n + 1 + 255) / 256 > 8 ? 8 : (n + 1 + 255) / 256, n);
    gather_rhs<<<grid, 256, 0, s>>>(c->G, c->cd, n, perm, W, ldw);
  }
  const int nrhs = n + 1;
  // forward substitution with unit lower L
  for (int i0 = 0; i0 < n; i0 += NB) {
    int jb = n - i0 < NB ? n - i0 : NB;
    trsm_block<true><<<(nrhs + 255) / 256, 256, 0, s>>>(LU + (size_t)i0 * ldw + i0, ldw, jb,
                                                         W + (size_t)i0 * ldw, ldw, nrhs);
    int rest = n - i0 - jb;
    if (rest > 0)
      gemm_sub(s, rest, nrhs, jb, LU + (size_t)(i0 + jb) * ldw + i0, ldw, W + (size_t)i0 * ldw, ldw,
               W + (size_t)(i0 + jb) * ldw, ldw);
  }
  // backward substitution with U
  int last = ((n - 1) / NB) * NB;
  for (int i0 = last; i0 >= 0; i0 -= NB) {
    int jb = n - i0 < NB ? n - i0 : NB;
    trsm_block<false><<<(nrhs + 255) / 256, 256, 0, s>>>(LU + (size_t)i0 * ldw + i0, ldw, jb,
                                                          W + (size_t)i0 * ldw, ldw, nrhs);
    if (i0 > 0)
      gemm_sub(s, i0, nrhs, jb, LU + i0, ldw, W + (size_t)i0 * ldw, ldw, W, ldw);
  }
  extract_diag_e<<<(n + 255) / 256, 256, 0, s>>>(W, n, ldw, diag, e);
  form_T<<<(n + 255) / 256, 256, 0, s>>>(W, n, ldw, c->God, v, n_o, T, c->L.ldt);
  form_o<<<1, 256, 0, s>>>(c->God, c->co, v, e, n, c->obj, ctl);
  return cuda_status(cudaGetLastError());
}

}  // namespace pngf
