// Tensor-core fold of the delayed set into the FP32 maintained inverse
// (mixed path), on the 5th-generation tensor cores of sm_103a:
//
//   W_lo[I, J] += sum_{i<r} alpha_i x_i[I] x_i[J]^T      (upper triangle of tiles)
//
// as real products with K = r: with Y = X diag(alpha),
//   Wr += Yr Xr^T - Yi Xi^T,   Wi += Yr Xi^T + Yi Xr^T.
// Each real product runs as 3xTF32: an operand is split into hi = tf32(a)
// and lo = a - hi, and hi.hi + hi.lo + lo.hi is accumulated in FP32 in tensor
// memory, which keeps the fold at FP32 accuracy (the rounding of W_lo itself).
//
// Data flow per tile (128 rows x 64 columns, both planes):
//   1. a prepare pass writes the split operands once per fold into global
//      images laid out exactly as the shared-memory tiles (K-major, no
//      swizzle: 8-row x 16-byte core matrices, 128 B apart along K, 1024 B
//      apart along the rows);
//   2. per K-chunk of 32, one bulk asynchronous copy (cp.async.bulk, the TMA
//      engine) per operand brings the images into shared memory, completing
//      an mbarrier transaction count;
//   3. one thread issues tcgen05.mma (kind::tf32, M = 128, N = 64, K = 8)
//      into two 64-column accumulators in tensor memory and commits to an
//      mbarrier;
//   4. the four warps read the accumulators back with tcgen05.ld, stage them
//      in shared memory and add them into W_lo with coalesced accesses.
// Every wait is bounded: on expiry the CTA latches PNGF_ETIMEOUT, waits
// (bounded) for what it issued, frees its tensor memory and returns.
#pragma once

#include "mixed_common.cuh"

namespace pngf {
namespace {

constexpr int TC_M = 128;            // rows of an output tile (MMA M)
constexpr int TC_N = 64;             // columns of an output tile (MMA N)
constexpr int TC_KC = 32;            // delayed columns per K-chunk
constexpr int TC_ASUB = TC_M * TC_KC * 4;  // one A sub-image (hi or lo, re or im): 16 KB
constexpr int TC_BSUB = TC_N * TC_KC * 4;  // one B sub-image: 8 KB
constexpr int TC_ACHUNK = 4 * TC_ASUB;     // Yr_hi, Yr_lo, Yi_hi, Yi_lo
constexpr int TC_BCHUNK = 4 * TC_BSUB;     // Xr_hi, Xr_lo, Xi_hi, Xi_lo
constexpr int TC_SMEM = TC_ACHUNK + TC_BCHUNK;  // 96 KB
constexpr int TC_TMEM_COLS = 128;               // Dr: columns 0..63, Di: 64..127
constexpr unsigned long long kTcSpin = 1ull << 22;

// byte offset of element (row, k) inside a K-major no-swizzle image of 32 K
__host__ __device__ __forceinline__ int tc_off(int row, int k) {
  return (row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float tf32_hi(float x) {
  unsigned u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// shared-memory matrix descriptor (K-major, no swizzle): start, LBO = 128 B
// between core matrices along K, SBO = 1024 B between 8-row groups, version 1
__device__ __forceinline__ unsigned long long tc_desc(unsigned smem_addr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((smem_addr & 0x3FFFF) >> 4);
  d |= (unsigned long long)(128 >> 4) << 16;
  d |= (unsigned long long)(1024 >> 4) << 32;
  d |= 1ull << 46;
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, K-major, N = 64, M = 128
__device__ __forceinline__ unsigned tc_idesc(bool negate_a) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((negate_a ? 1u : 0u) << 13) | ((unsigned)(TC_N >> 3) << 17) |
         ((unsigned)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(unsigned mb, unsigned phase) {
  for (unsigned long long it = 0; it < kTcSpin; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(mb), "r"(phase)
        : "memory");
    if (ok) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

// number of tiles (128-row block ti, 64-column block tj >= 2 ti) and the tile of index t
__device__ __forceinline__ long long tc_tiles(int n) {
  const int nI = (n + TC_M - 1) / TC_M, nJ = (n + TC_N - 1) / TC_N;
  long long T = 0;
  for (int ti = 0; ti < nI; ++ti) T += max(0, nJ - 2 * ti);
  return T;
}
__device__ __forceinline__ void tc_tile(long long t, int n, int& ti, int& tj) {
  const int nI = (n + TC_M - 1) / TC_M, nJ = (n + TC_N - 1) / TC_N;
  for (ti = 0; ti < nI; ++ti) {
    long long cnt = max(0, nJ - 2 * ti);
    if (t < cnt) {
      tj = 2 * ti + (int)t;
      return;
    }
    t -= cnt;
  }
  ti = tj = 0;
}

// Prepare pass (all threads of the calling grid, elements split round-robin):
// split images of Y = X diag(alpha) (A side, 128-row blocks) and X (B side,
// 64-row blocks), for nk = ceil(r / 32) chunks, zero-padded past n and r.
__device__ __noinline__ void tc_prepare(const SweepArgs& a, int r, unsigned char* imgA, unsigned char* imgB, long long gtid,
                           long long gstride) {
  const int n = a.n, nk = (r + TC_KC - 1) / TC_KC;
  const int nI = (n + TC_M - 1) / TC_M, nJ = (n + TC_N - 1) / TC_N;
  // A side
  const long long totA = (long long)nI * TC_M * nk * TC_KC;
  for (long long e = gtid; e < totA; e += gstride) {
    const int k = (int)(e % TC_KC);
    long long rest = e / TC_KC;
    const int row = (int)(rest % TC_M);
    rest /= TC_M;
    const int c = (int)(rest % nk);
    const int I = (int)(rest / nk);
    const int gi = I * TC_M + row, q = c * TC_KC + k;
    float yr = 0.f, yi = 0.f;
    if (gi < n && q < r) {
      c128 al = a.xa[q];
      float2 x = a.X[(size_t)gi * a.R + q];
      float ax = (float)al.x, ay = (float)al.y;
      yr = fmaf(ax, x.x, -ay * x.y);
      yi = fmaf(ax, x.y, ay * x.x);
    }
    unsigned char* base = imgA + ((size_t)I * nk + c) * TC_ACHUNK + tc_off(row, k);
    float yr_hi = tf32_hi(yr), yi_hi = tf32_hi(yi);
    *reinterpret_cast<float*>(base + 0 * TC_ASUB) = yr_hi;
    *reinterpret_cast<float*>(base + 1 * TC_ASUB) = yr - yr_hi;
    *reinterpret_cast<float*>(base + 2 * TC_ASUB) = yi_hi;
    *reinterpret_cast<float*>(base + 3 * TC_ASUB) = yi - yi_hi;
  }
  // B side
  const long long totB = (long long)nJ * TC_N * nk * TC_KC;
  for (long long e = gtid; e < totB; e += gstride) {
    const int k = (int)(e % TC_KC);
    long long rest = e / TC_KC;
    const int row = (int)(rest % TC_N);
    rest /= TC_N;
    const int c = (int)(rest % nk);
    const int J = (int)(rest / nk);
    const int gj = J * TC_N + row, q = c * TC_KC + k;
    float xr = 0.f, xi = 0.f;
    if (gj < n && q < r) {
      float2 x = a.X[(size_t)gj * a.R + q];
      xr = x.x;
      xi = x.y;
    }
    unsigned char* base = imgB + ((size_t)J * nk + c) * TC_BCHUNK + tc_off(row, k);
    float xr_hi = tf32_hi(xr), xi_hi = tf32_hi(xi);
    *reinterpret_cast<float*>(base + 0 * TC_BSUB) = xr_hi;
    *reinterpret_cast<float*>(base + 1 * TC_BSUB) = xr - xr_hi;
    *reinterpret_cast<float*>(base + 2 * TC_BSUB) = xi_hi;
    *reinterpret_cast<float*>(base + 3 * TC_BSUB) = xi - xi_hi;
  }
  // the images are read next by bulk asynchronous copies (async proxy)
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

struct TcState {
  unsigned tmem;     // tensor-memory base address of this CTA's accumulators
  unsigned mb_load;  // mbarrier: bulk copies landed
  unsigned mb_mma;   // mbarrier: MMAs of a chunk complete
  unsigned ph_load, ph_mma;
};

// Tiles [t_begin, T) with step t_step, by the first 128 threads of the CTA
// (warp w reads accumulator lanes 32w..32w+31).  Returns false after a timeout.
__device__ bool tc_fold_tiles(const SweepArgs& a, int r, const unsigned char* imgA, const unsigned char* imgB,
                              unsigned char* smem, TcState& st, long long t_begin, long long t_step) {
  const int n = a.n, nk = (r + TC_KC - 1) / TC_KC;
  const long long T = tc_tiles(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned sA = (unsigned)__cvta_generic_to_shared(smem);
  const unsigned sB = sA + TC_ACHUNK;
  __shared__ int s_fail;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (long long t = t_begin; t < T; t += t_step) {
    int ti, tj;
    tc_tile(t, n, ti, tj);
    for (int c = 0; c < nk; ++c) {
      if (tid == 0) {
        const unsigned char* ga = imgA + ((size_t)ti * nk + c) * TC_ACHUNK;
        const unsigned char* gb = imgB + ((size_t)tj * nk + c) * TC_BCHUNK;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(st.mb_load), "r"(TC_SMEM)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sA),
                     "l"(ga), "r"(TC_ACHUNK), "r"(st.mb_load)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sB),
                     "l"(gb), "r"(TC_BCHUNK), "r"(st.mb_load)
                     : "memory");
      }
      if (tid < 128 && !mbar_wait(st.mb_load, st.ph_load)) s_fail = 1;
      st.ph_load ^= 1;
      __syncthreads();
      if (s_fail) return false;
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const unsigned dR = st.tmem, dI = st.tmem + TC_N;
        const unsigned id_pos = tc_idesc(false), id_neg = tc_idesc(true);
#pragma unroll
        for (int ks = 0; ks < TC_KC / 8; ++ks) {
          const unsigned ko = 256u * ks;
          const unsigned long long yr_hi = tc_desc(sA + 0 * TC_ASUB + ko), yr_lo = tc_desc(sA + 1 * TC_ASUB + ko);
          const unsigned long long yi_hi = tc_desc(sA + 2 * TC_ASUB + ko), yi_lo = tc_desc(sA + 3 * TC_ASUB + ko);
          const unsigned long long xr_hi = tc_desc(sB + 0 * TC_BSUB + ko), xr_lo = tc_desc(sB + 1 * TC_BSUB + ko);
          const unsigned long long xi_hi = tc_desc(sB + 2 * TC_BSUB + ko), xi_lo = tc_desc(sB + 3 * TC_BSUB + ko);
          const unsigned first = (c == 0 && ks == 0) ? 0u : 1u;
          // Wr += Yr Xr^T - Yi Xi^T
          tc_mma(dR, yr_hi, xr_hi, id_pos, first);
          tc_mma(dR, yr_hi, xr_lo, id_pos, 1);
          tc_mma(dR, yr_lo, xr_hi, id_pos, 1);
          tc_mma(dR, yi_hi, xi_hi, id_neg, 1);
          tc_mma(dR, yi_hi, xi_lo, id_neg, 1);
          tc_mma(dR, yi_lo, xi_hi, id_neg, 1);
          // Wi += Yr Xi^T + Yi Xr^T
          tc_mma(dI, yr_hi, xi_hi, id_pos, first);
          tc_mma(dI, yr_hi, xi_lo, id_pos, 1);
          tc_mma(dI, yr_lo, xi_hi, id_pos, 1);
          tc_mma(dI, yi_hi, xr_hi, id_pos, 1);
          tc_mma(dI, yi_hi, xr_lo, id_pos, 1);
          tc_mma(dI, yi_lo, xr_hi, id_pos, 1);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(st.mb_mma)
                     : "memory");
      }
      if (tid < 128 && !mbar_wait(st.mb_mma, st.ph_mma)) s_fail = 1;
      st.ph_mma ^= 1;
      __syncthreads();
      if (s_fail) return false;
    }
    // epilogue: accumulators -> shared staging -> W_lo (coalesced read-modify-write)
    asm volatile("tcgen05.fence::after_thread_sync;");
    float* stage = reinterpret_cast<float*>(smem);  // [2][128][65]
    if (tid < 128) {
      const unsigned lane_base = (unsigned)(32 * warp) << 16;
#pragma unroll
      for (int half = 0; half < 4; ++half) {  // Dr cols 0-31, 32-63, Di cols 64-95, 96-127
        unsigned v[32];
        const unsigned addr = st.tmem + lane_base + 32u * half;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
              "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        const int plane = half >> 1, col0 = 32 * (half & 1);
        const int row = 32 * warp + lane;
#pragma unroll
        for (int q = 0; q < 32; ++q) stage[(plane * TC_M + row) * (TC_N + 1) + col0 + q] = __uint_as_float(v[q]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    {
      // 16-byte accesses, all loads of a thread issued before its stores
      const int i0 = ti * TC_M, j0 = tj * TC_N;
      const int nthr = (int)blockDim.x;
      constexpr int V = 4, PER_ROW = TC_N / V, ITEMS = TC_M * PER_ROW;  // float4 items per plane
      if (tid < nthr) {
        for (int base = tid; base < ITEMS; base += nthr * 8) {
          float4 wr[8], wi[8];
          int ok[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int it = base + u * nthr;
            const int row = it / PER_ROW, col = (it % PER_ROW) * V;
            const int gi = i0 + row, gj = j0 + col;
            ok[u] = (it < ITEMS && gi < n) ? (gj + V <= n ? 2 : (gj < n ? 1 : 0)) : 0;
            if (ok[u] == 2) {
              size_t o = (size_t)gi * a.ldl + gj;
              wr[u] = *reinterpret_cast<const float4*>(a.Wr + o);
              wi[u] = *reinterpret_cast<const float4*>(a.Wi + o);
            }
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int it = base + u * nthr;
            if (!ok[u]) continue;
            const int row = it / PER_ROW, col = (it % PER_ROW) * V;
            const int gi = i0 + row, gj = j0 + col;
            const float* sr = stage + (0 * TC_M + row) * (TC_N + 1) + col;
            const float* si = stage + (1 * TC_M + row) * (TC_N + 1) + col;
            size_t o = (size_t)gi * a.ldl + gj;
            if (ok[u] == 2) {
              wr[u].x += sr[0]; wr[u].y += sr[1]; wr[u].z += sr[2]; wr[u].w += sr[3];
              wi[u].x += si[0]; wi[u].y += si[1]; wi[u].z += si[2]; wi[u].w += si[3];
              *reinterpret_cast<float4*>(a.Wr + o) = wr[u];
              *reinterpret_cast<float4*>(a.Wi + o) = wi[u];
            } else {
              for (int q = 0; q < V && gj + q < n; ++q) {
                a.Wr[o + q] += sr[q];
                a.Wi[o + q] += si[q];
              }
            }
          }
        }
      }
    }
    // the next tile's bulk copies (async proxy) overwrite the staging area
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
  return true;
}

// tensor memory of the CTA: warp 0 allocates TC_TMEM_COLS columns
__device__ __forceinline__ void tc_alloc(unsigned* slot) {
  if (threadIdx.x < 32) {
    unsigned s = (unsigned)__cvta_generic_to_shared(slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s), "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
}
__device__ __forceinline__ void tc_free(unsigned tmem) {
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}
__device__ __forceinline__ void tc_mbar_init(unsigned long long* mb_load, unsigned long long* mb_mma) {
  if (threadIdx.x == 0) {
    unsigned a = (unsigned)__cvta_generic_to_shared(mb_load), b = (unsigned)__cvta_generic_to_shared(mb_mma);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
}

// bytes of the global operand images for a region of n pixels and r <= R delayed columns
__host__ __device__ __forceinline__ size_t tc_image_bytes(int n, int R) {
  const size_t nk = (size_t)(R + TC_KC - 1) / TC_KC;
  const size_t nI = (size_t)(n + TC_M - 1) / TC_M, nJ = (size_t)(n + TC_N - 1) / TC_N;
  return nI * nk * TC_ACHUNK + nJ * nk * TC_BCHUNK;
}

}  // namespace
}  // namespace pngf
