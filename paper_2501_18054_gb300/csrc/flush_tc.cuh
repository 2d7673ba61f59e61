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
//   2. per K-chunk of 16, one bulk asynchronous copy (cp.async.bulk, the TMA
//      engine) per operand brings the images into one of two shared-memory
//      buffers, completing that buffer's mbarrier transaction count; the copy
//      of chunk c + 1 runs while the tensor cores work on chunk c;
//   3. one thread issues tcgen05.mma (kind::tf32, M = 128, N = 64, K = 8)
//      into two 64-column accumulators in tensor memory and commits to the
//      buffer's MMA mbarrier;
//   4. the tile of W_lo is read into registers when the tile starts; four
//      warps read the accumulators back with tcgen05.ld and stage them in
//      shared memory, and every thread adds them into its part of the tile.
// Every wait is bounded: on expiry the CTA latches PNGF_ETIMEOUT, waits
// (bounded) for what it issued, frees its tensor memory and returns.
#pragma once

#include "mixed_common.cuh"

namespace pngf {
namespace {

constexpr int TC_M = 128;            // rows of an output tile (MMA M)
constexpr int TC_N = 64;             // columns of an output tile (MMA N)
constexpr int TC_KC = 16;            // delayed columns per K-chunk
constexpr int TC_ASUB = TC_M * TC_KC * 4;  // one A sub-image (hi or lo, re or im): 16 KB
constexpr int TC_BSUB = TC_N * TC_KC * 4;  // one B sub-image: 8 KB
constexpr int TC_ACHUNK = 4 * TC_ASUB;     // Yr_hi, Yr_lo, Yi_hi, Yi_lo
constexpr int TC_BCHUNK = 4 * TC_BSUB;     // Xr_hi, Xr_lo, Xi_hi, Xi_lo
constexpr int TC_BUF = TC_ACHUNK + TC_BCHUNK;   // one buffer: 48 KB
constexpr int TC_SMEM = 2 * TC_BUF;             // two buffers: 96 KB
constexpr int TC_TMEM_COLS = 128;               // Dr: columns 0..63, Di: 64..127
constexpr unsigned long long kTcSpin = 1ull << 22;

// byte offset of element (row, k) inside a K-major no-swizzle image of TC_KC
// columns: 8-row x 16-byte core matrices, 128 B apart along K, TC_SBO apart
// along the rows
constexpr int TC_SBO = TC_KC / 4 * 128;
__host__ __device__ __forceinline__ int tc_off(int row, int k) {
  return (row >> 3) * TC_SBO + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float tf32_hi(float x) {
  unsigned u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// shared-memory matrix descriptor (K-major, no swizzle): start, LBO = 128 B
// between core matrices along K, SBO = TC_SBO between 8-row groups, version 1
__device__ __forceinline__ unsigned long long tc_desc(unsigned smem_addr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((smem_addr & 0x3FFFF) >> 4);
  d |= (unsigned long long)(128 >> 4) << 16;
  d |= (unsigned long long)(TC_SBO >> 4) << 32;
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

// four consecutive k of one core-matrix row (16 bytes) in the four
// sub-images re_hi, re_lo, im_hi, im_lo (sub apart)
__device__ __forceinline__ void tc_store_split(unsigned char* base, int sub, const float re[4], const float im[4]) {
  float4 h, l;
  h.x = tf32_hi(re[0]); h.y = tf32_hi(re[1]); h.z = tf32_hi(re[2]); h.w = tf32_hi(re[3]);
  l.x = re[0] - h.x; l.y = re[1] - h.y; l.z = re[2] - h.z; l.w = re[3] - h.w;
  *reinterpret_cast<float4*>(base + 0 * sub) = h;
  *reinterpret_cast<float4*>(base + 1 * sub) = l;
  h.x = tf32_hi(im[0]); h.y = tf32_hi(im[1]); h.z = tf32_hi(im[2]); h.w = tf32_hi(im[3]);
  l.x = im[0] - h.x; l.y = im[1] - h.y; l.z = im[2] - h.z; l.w = im[3] - h.w;
  *reinterpret_cast<float4*>(base + 2 * sub) = h;
  *reinterpret_cast<float4*>(base + 3 * sub) = l;
}

// Prepare pass (all threads of the calling grid, items split round-robin):
// split images of Y = X diag(alpha) (A side, 128-row blocks) and X (B side,
// 64-row blocks), for nk = ceil(r / TC_KC) chunks, zero-padded past n and r.
// An item is four consecutive delayed columns of one row: one 32-byte read of
// X and one 16-byte write per sub-image (four k of a core-matrix row).
__device__ __noinline__ void tc_prepare(const SweepArgs& a, int r, unsigned char* imgA, unsigned char* imgB,
                                        long long gtid, long long gstride) {
  __shared__ float2 s_al[kMaxDelay];
  for (int q = threadIdx.x; q < r; q += blockDim.x) {
    const c128 al = a.xa[q];
    s_al[q] = make_float2((float)al.x, (float)al.y);
  }
  __syncthreads();
  const int n = a.n, nk = (r + TC_KC - 1) / TC_KC;
  const unsigned nI = (unsigned)(n + TC_M - 1) / TC_M, nJ = (unsigned)(n + TC_N - 1) / TC_N;
  constexpr unsigned KQ = TC_KC / 4;  // items per chunk row
  // A side: item = ((I * nk + c) * TC_M + row) * KQ + kq
  const unsigned totA = nI * (unsigned)nk * TC_M * KQ;
  for (unsigned e = (unsigned)gtid; e < totA; e += (unsigned)gstride) {
    const unsigned kq = e % KQ, row = (e / KQ) % TC_M, rest = e / (KQ * TC_M);
    const unsigned c = rest % (unsigned)nk, I = rest / (unsigned)nk;
    const int gi = (int)(I * TC_M + row), q0 = (int)(c * TC_KC + kq * 4);
    float yr[4], yi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      yr[u] = yi[u] = 0.f;
      const int q = q0 + u;
      if (gi < n && q < r) {
        const float2 x = a.X[(size_t)gi * a.R + q], al = s_al[q];
        yr[u] = fmaf(al.x, x.x, -al.y * x.y);
        yi[u] = fmaf(al.x, x.y, al.y * x.x);
      }
    }
    unsigned char* base = imgA + ((size_t)I * nk + c) * TC_ACHUNK + tc_off((int)row, (int)kq * 4);
    tc_store_split(base, TC_ASUB, yr, yi);
  }
  // B side: item = ((J * nk + c) * TC_N + row) * KQ + kq
  const unsigned totB = nJ * (unsigned)nk * TC_N * KQ;
  for (unsigned e = (unsigned)gtid; e < totB; e += (unsigned)gstride) {
    const unsigned kq = e % KQ, row = (e / KQ) % TC_N, rest = e / (KQ * TC_N);
    const unsigned c = rest % (unsigned)nk, J = rest / (unsigned)nk;
    const int gj = (int)(J * TC_N + row), q0 = (int)(c * TC_KC + kq * 4);
    float xr[4], xi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      xr[u] = xi[u] = 0.f;
      const int q = q0 + u;
      if (gj < n && q < r) {
        const float2 x = a.X[(size_t)gj * a.R + q];
        xr[u] = x.x;
        xi[u] = x.y;
      }
    }
    unsigned char* base = imgB + ((size_t)J * nk + c) * TC_BCHUNK + tc_off((int)row, (int)kq * 4);
    tc_store_split(base, TC_BSUB, xr, xi);
  }
  // the images are read next by bulk asynchronous copies (async proxy)
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Tensor-core state of a CTA.  Barriers 0, 1: operand copies into buffer 0, 1;
// barriers 2, 3: MMA commits that read buffer 0, 1.  Only thread 0 issues and
// waits: ph is the parity of the next wait, pend marks an issued operation
// that has not been waited for.
struct TcState {
  unsigned tmem;  // tensor-memory base address of this CTA's accumulators
  unsigned mb[4];
  unsigned ph[4];
  int pend[4];
};

// all threads: barriers (thread 0), tensor memory (warp 0), then a CTA barrier
__device__ __forceinline__ void tc_setup(TcState& st, unsigned long long* bars, unsigned* tmem_slot) {
  if (threadIdx.x == 0) {
    for (int q = 0; q < 4; ++q) {
      const unsigned m = (unsigned)__cvta_generic_to_shared(bars + q);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(m));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (threadIdx.x < 32) {
    const unsigned sl = (unsigned)__cvta_generic_to_shared(tmem_slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sl), "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  st.tmem = *tmem_slot;
  for (int q = 0; q < 4; ++q) {
    st.mb[q] = (unsigned)__cvta_generic_to_shared(bars + q);
    st.ph[q] = 0;
    st.pend[q] = 0;
  }
}

// thread 0: wait (bounded) for barrier q's pending operation; false on expiry
__device__ __forceinline__ bool tc_wait(TcState& st, int q) {
  if (!st.pend[q]) return true;
  if (!mbar_wait(st.mb[q], st.ph[q])) return false;
  st.ph[q] ^= 1;
  st.pend[q] = 0;
  return true;
}

// all threads: after a failure thread 0 gives what it issued a bounded time to
// land (copies first, then the MMA commits), then warp 0 frees the tensor memory
__device__ __forceinline__ void tc_teardown(TcState& st, bool failed) {
  if (failed && threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) tc_wait(st, q);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(st.tmem), "r"(TC_TMEM_COLS));
}

// thread 0: bulk copies of K-chunk c of tile (ti, tj) into buffer bf
__device__ __forceinline__ void tc_issue_copy(TcState& st, int bf, unsigned sbuf, const unsigned char* imgA,
                                              const unsigned char* imgB, int ti, int tj, int c, int nk) {
  const unsigned char* ga = imgA + ((size_t)ti * nk + c) * TC_ACHUNK;
  const unsigned char* gb = imgB + ((size_t)tj * nk + c) * TC_BCHUNK;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(st.mb[bf]), "r"(TC_BUF) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sbuf),
               "l"(ga), "r"(TC_ACHUNK), "r"(st.mb[bf])
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   sbuf + TC_ACHUNK),
               "l"(gb), "r"(TC_BCHUNK), "r"(st.mb[bf])
               : "memory");
  st.pend[bf] = 1;
}

// thread 0: the 3xTF32 products of one K-chunk in buffer sbuf, committed to barrier 2 + bf
__device__ __forceinline__ void tc_issue_mma(TcState& st, int bf, unsigned sbuf, bool first_chunk) {
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned sA = sbuf, sB = sbuf + TC_ACHUNK;
  const unsigned dR = st.tmem, dI = st.tmem + TC_N;
  const unsigned id_pos = tc_idesc(false), id_neg = tc_idesc(true);
#pragma unroll
  for (int ks = 0; ks < TC_KC / 8; ++ks) {
    const unsigned ko = 256u * ks;
    const unsigned long long yr_hi = tc_desc(sA + 0 * TC_ASUB + ko), yr_lo = tc_desc(sA + 1 * TC_ASUB + ko);
    const unsigned long long yi_hi = tc_desc(sA + 2 * TC_ASUB + ko), yi_lo = tc_desc(sA + 3 * TC_ASUB + ko);
    const unsigned long long xr_hi = tc_desc(sB + 0 * TC_BSUB + ko), xr_lo = tc_desc(sB + 1 * TC_BSUB + ko);
    const unsigned long long xi_hi = tc_desc(sB + 2 * TC_BSUB + ko), xi_lo = tc_desc(sB + 3 * TC_BSUB + ko);
    const unsigned first = (first_chunk && ks == 0) ? 0u : 1u;
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
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(st.mb[2 + bf])
               : "memory");
  st.pend[2 + bf] = 1;
}

// Tiles [t_begin, T) with step t_step; thread 0 drives the copies and the
// MMAs, the first 128 threads read the accumulators (warp w: lanes
// 32w..32w+31), all threads (at least 256) read and write the tile of W_lo.
// smem: TC_SMEM bytes.  Returns false after a timeout (the caller then calls
// tc_teardown with failed = true).
__device__ bool tc_fold_tiles(const SweepArgs& a, int r, const unsigned char* imgA, const unsigned char* imgB,
                              unsigned char* smem, TcState& st, long long t_begin, long long t_step) {
  const int n = a.n, nk = (r + TC_KC - 1) / TC_KC;
  const long long T = tc_tiles(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned s0 = (unsigned)__cvta_generic_to_shared(smem);
  __shared__ int s_fail;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  // epilogue items: float4 groups of the 128 x 64 tile, item it = row * 16 + column / 4
  constexpr int V = 4, PER_ROW = TC_N / V, ITEMS = TC_M * PER_ROW, MAXU = 8;
  const int nthr = (int)blockDim.x;
  if (nthr * MAXU < ITEMS) return false;  // every item needs a thread slot (>= 256 threads)
  for (long long t = t_begin; t < T; t += t_step) {
    int ti, tj;
    tc_tile(t, n, ti, tj);
    const int i0 = ti * TC_M, j0 = tj * TC_N;
    if (tid == 0) {
      // chunk c in buffer c & 1; the copy of chunk c + 1 is issued once the
      // MMAs of chunk c - 1 (same buffer) have completed
      bool ok = true;
      tc_issue_copy(st, 0, s0, imgA, imgB, ti, tj, 0, nk);
      for (int c = 0; c < nk && ok; ++c) {
        const int bf = c & 1;
        if (c + 1 < nk) {
          ok = tc_wait(st, 2 + (bf ^ 1));
          if (ok) tc_issue_copy(st, bf ^ 1, s0 + (bf ^ 1) * TC_BUF, imgA, imgB, ti, tj, c + 1, nk);
        }
        if (ok) ok = tc_wait(st, bf);
        if (ok) tc_issue_mma(st, bf, s0 + bf * TC_BUF, c == 0);
      }
      // the commits complete in order: chunk nk - 2's barrier, then nk - 1's
      if (ok && nk >= 2) ok = tc_wait(st, 2 + ((nk - 2) & 1));
      if (ok) ok = tc_wait(st, 2 + ((nk - 1) & 1));
      if (!ok) s_fail = 1;
    }
    // the tile of W_lo is read now, while the copies and the MMAs run
    float4 wr[MAXU], wi[MAXU];
    int okv[MAXU];
#pragma unroll
    for (int u = 0; u < MAXU; ++u) {
      const int it = tid + u * nthr;
      const int row = it / PER_ROW, col = (it % PER_ROW) * V;
      const int gi = i0 + row, gj = j0 + col;
      okv[u] = (it < ITEMS && gi < n) ? (gj + V <= n ? 2 : (gj < n ? 1 : 0)) : 0;
      if (okv[u] == 2) {
        const size_t o = (size_t)gi * a.ldl + gj;
        wr[u] = *reinterpret_cast<const float4*>(a.Wr + o);
        wi[u] = *reinterpret_cast<const float4*>(a.Wi + o);
      }
    }
    __syncthreads();
    if (s_fail) return false;
    // epilogue: accumulators -> shared staging -> W_lo
    asm volatile("tcgen05.fence::after_thread_sync;");
    float* stage = reinterpret_cast<float*>(smem);  // [2][128][65], over the consumed buffers
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
    // add the accumulators to the prefetched tile and store it
#pragma unroll
    for (int u = 0; u < MAXU; ++u) {
      const int it = tid + u * nthr;
      if (!okv[u]) continue;
      const int row = it / PER_ROW, col = (it % PER_ROW) * V;
      const int gi = i0 + row, gj = j0 + col;
      const float* sr = stage + (0 * TC_M + row) * (TC_N + 1) + col;
      const float* si = stage + (1 * TC_M + row) * (TC_N + 1) + col;
      const size_t o = (size_t)gi * a.ldl + gj;
      if (okv[u] == 2) {
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
    // the next tile's bulk copies (async proxy) overwrite the staging area
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
  return true;
}

// bytes of the global operand images for a region of n pixels and r <= R delayed columns
__host__ __device__ __forceinline__ size_t tc_image_bytes(int n, int R) {
  const size_t nk = (size_t)(R + TC_KC - 1) / TC_KC;
  const size_t nI = (size_t)(n + TC_M - 1) / TC_M, nJ = (size_t)(n + TC_N - 1) / TC_N;
  return nI * nk * TC_ACHUNK + nJ * nk * TC_BCHUNK;
}

}  // namespace
}  // namespace pngf
