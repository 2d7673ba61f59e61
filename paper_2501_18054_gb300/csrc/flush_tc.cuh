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
// Data flow per tile (128 rows x 64 NB columns, both planes; NB = 2 for the
// persistent search, 1 for the batch kernel):
//   1. a prepare pass writes the split operands once per fold into global
//      images laid out exactly as the shared-memory tiles (K-major, no
//      swizzle: 8-row x 16-byte core matrices, 128 B apart along K, 512 B
//      apart along the rows), in blocks of 128 rows for both operands;
//   2. per K-chunk of 16, one bulk asynchronous copy (cp.async.bulk, the TMA
//      engine) per operand brings the images into one of two shared-memory
//      buffers, completing that buffer's mbarrier transaction count; the copy
//      of chunk c + 1 runs while the tensor cores work on chunk c;
//   3. one thread issues tcgen05.mma (kind::tf32, M = 128, N = 64 NB, K = 8:
//      twelve per K-step, the 3xTF32 terms of the four real products) into
//      the tile's accumulator in tensor memory (Dr and Di, 64 NB columns
//      each) and commits to the buffer's MMA mbarrier;
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
constexpr int TC_N = 128;            // rows of a B image block (a tile covers 64 NB of them)
constexpr int TC_KC = 16;            // delayed columns per K-chunk
constexpr int TC_ASUB = TC_M * TC_KC * 4;  // one A sub-image (hi or lo, re or im): 8 KB
constexpr int TC_BSUB = TC_N * TC_KC * 4;  // one B sub-image of a global block: 8 KB
constexpr int TC_ACHUNK = 4 * TC_ASUB;     // Yr_hi, Yr_lo, Yi_hi, Yi_lo
constexpr int TC_BCHUNK = 4 * TC_BSUB;     // Xr_hi, Xr_lo, Xi_hi, Xi_lo
constexpr int TC_NBUF = 2;                      // operand buffers
constexpr int TC_PREF = 1;                      // chunks copied ahead of the one multiplied
constexpr int TC_PC = 16;                       // tile columns per epilogue part
constexpr int TC_STAGE = 2 * TC_M * TC_PC * 4;  // one part of both planes: 16 KB
// A tile of the fold is 128 rows x 64 NB columns: one 128-row block of Y (A
// operand) against 64 NB rows of X (B operand, the whole of a 128-row image
// block for NB = 2, one half of it for NB = 1), NB = 1 or 2.
__host__ __device__ constexpr int tc_tile_cols(int nb) { return 64 * nb; }
__host__ __device__ constexpr int tc_bsub_smem(int nb) { return tc_tile_cols(nb) * TC_KC * 4; }  // 4 / 8 KB
__host__ __device__ constexpr int tc_buf_bytes(int nb) { return TC_ACHUNK + 4 * tc_bsub_smem(nb); }  // 48 / 64 KB
// float4 slot of stage row `row`, column group q4 (4 columns): the XOR spreads
// both the row-per-lane writes and the row-contiguous reads over all banks
__device__ __forceinline__ int tc_stage_slot(int row, int q4) { return row * 4 + (q4 ^ ((row >> 1) & 3)); }
__host__ __device__ constexpr int tc_fold_smem(int nb) { return TC_NBUF * tc_buf_bytes(nb) + TC_STAGE; }
// tensor memory: two accumulators of (Dr: 64 NB columns, Di: 64 NB columns)
__host__ __device__ constexpr int tc_tmem_cols(int nb) { return 2 * 128 * nb; }
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

// instruction descriptor: D = F32, A = B = TF32, K-major, N = n_cols, M = 128
__device__ __forceinline__ unsigned tc_idesc(bool negate_a, int n_cols) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((negate_a ? 1u : 0u) << 13) | ((unsigned)(n_cols >> 3) << 17) |
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

// 128-row blocks of the B image
__host__ __device__ __forceinline__ int tc_njb(int n) { return (n + TC_N - 1) / TC_N; }

// number of tiles of the upper triangle (128-row block ti, 64 NB-column block
// tj >= 2 ti / NB) and the tile of index t
template <int NB>
__device__ __forceinline__ long long tc_tiles(int n) {
  static_assert(NB == 1 || NB == 2, "tiles of 128 x 64 or 128 x 128");
  const int nI = (n + TC_M - 1) / TC_M, nJ = (n + tc_tile_cols(NB) - 1) / tc_tile_cols(NB);
  long long T = 0;
  for (int ti = 0; ti < nI; ++ti) T += max(0, nJ - 2 * ti / NB);
  return T;
}
template <int NB>
__device__ __forceinline__ void tc_tile(long long t, int n, int& ti, int& tj) {
  const int nI = (n + TC_M - 1) / TC_M, nJ = (n + tc_tile_cols(NB) - 1) / tc_tile_cols(NB);
  for (ti = 0; ti < nI; ++ti) {
    long long cnt = max(0, nJ - 2 * ti / NB);
    if (t < cnt) {
      tj = 2 * ti / NB + (int)t;
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
// split images of Y = X diag(alpha) (A side) and X (B side), both in 128-row
// blocks, for nk = ceil(r / TC_KC) chunks, zero-padded past n and r.
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
  const unsigned nI = (unsigned)(n + TC_M - 1) / TC_M, nJ = (unsigned)tc_njb(n);
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

// Tensor-core state of a CTA, kept across calls of tc_fold_tiles.  Barriers
// (index): TC_B_LOAD + b operand copies landed in buffer b; TC_B_FREE + b the
// MMAs reading buffer b completed; TC_B_FULL + a accumulator a complete;
// TC_B_EMPTY + a accumulator a read back (one arrival per epilogue warp).  ph
// is the parity of a thread's next wait on a barrier (each role waits on its
// own barriers, and every phase of those is waited for exactly once, so the
// parities stay in step across calls); pend marks a phase the producer
// expects and has not yet waited for.
constexpr int TC_B_LOAD = 0, TC_B_FREE = TC_NBUF, TC_B_FULL = 2 * TC_NBUF, TC_B_EMPTY = 2 * TC_NBUF + 2;
constexpr int TC_NBAR = 2 * TC_NBUF + 4;
struct TcState {
  unsigned tmem;       // tensor-memory base address: accumulator a at columns a tmem_cols / 2 ..
  unsigned tmem_cols;  // columns allocated: tc_tmem_cols(NB) of the fold that uses them
  unsigned mb[TC_NBAR];
  unsigned ph[TC_NBAR];
  int pend[TC_NBAR];
};

// epilogue warps: the last 8 warps of a CTA of at least 16 warps (two per
// tensor-memory lane quadrant), else the last 4 (one per quadrant)
__device__ __forceinline__ int tc_epi_warps() { return (blockDim.x >> 5) >= 16 ? 8 : 4; }

// all threads: barriers (thread 0), tensor memory (warp 0), then a CTA barrier
__device__ __forceinline__ void tc_setup(TcState& st, unsigned long long* bars, unsigned* tmem_slot, int tmem_cols) {
  if (threadIdx.x == 0) {
    for (int q = 0; q < TC_NBAR; ++q) {
      const unsigned m = (unsigned)__cvta_generic_to_shared(bars + q);
      const unsigned count = q >= TC_B_EMPTY ? (unsigned)tc_epi_warps() : 1u;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(m), "r"(count));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (threadIdx.x < 32) {
    const unsigned sl = (unsigned)__cvta_generic_to_shared(tmem_slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sl), "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  st.tmem = *tmem_slot;
  st.tmem_cols = (unsigned)tmem_cols;
  for (int q = 0; q < TC_NBAR; ++q) {
    st.mb[q] = (unsigned)__cvta_generic_to_shared(bars + q);
    st.ph[q] = 0;
    st.pend[q] = 0;
  }
}

// wait (bounded) for the next phase of barrier q; false on expiry
__device__ __forceinline__ bool tc_wait_phase(TcState& st, int q) {
  if (!mbar_wait(st.mb[q], st.ph[q])) return false;
  st.ph[q] ^= 1;
  return true;
}
// producer: wait for barrier q's pending operation, if any
__device__ __forceinline__ bool tc_wait(TcState& st, int q) {
  if (!st.pend[q]) return true;
  if (!tc_wait_phase(st, q)) return false;
  st.pend[q] = 0;
  return true;
}

// all threads: after a failure thread 0 gives what it issued a bounded time to
// land (copies, then the MMA commits), then warp 0 frees the tensor memory
__device__ __forceinline__ void tc_teardown(TcState& st, bool failed) {
  if (failed && threadIdx.x == 0)
    for (int q = 0; q < TC_B_FULL; ++q) tc_wait(st, q);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(st.tmem), "r"(st.tmem_cols));
}

// producer: bulk copies of K-chunk c of tile (ti, tj) into buffer bf: the A
// chunk of row block ti, then the B chunk of the tile's 64 NB columns (NB = 2:
// image block tj in one copy; NB = 1: half tj & 1 of image block tj / 2, one
// copy per sub-image)
template <int NB>
__device__ __forceinline__ void tc_issue_copy(TcState& st, int bf, unsigned sbuf, const unsigned char* imgA,
                                              const unsigned char* imgB, int ti, int tj, int c, int nk) {
  const unsigned mb = st.mb[TC_B_LOAD + bf];
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(tc_buf_bytes(NB)) : "memory");
  const unsigned char* ga = imgA + ((size_t)ti * nk + c) * TC_ACHUNK;
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sbuf),
               "l"(ga), "r"(TC_ACHUNK), "r"(mb)
               : "memory");
  if (NB == 2) {
    const unsigned char* gb = imgB + ((size_t)tj * nk + c) * TC_BCHUNK;
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sbuf + TC_ACHUNK),
                 "l"(gb), "r"(TC_BCHUNK), "r"(mb)
                 : "memory");
  } else {
    const unsigned char* gb = imgB + ((size_t)(tj >> 1) * nk + c) * TC_BCHUNK + (size_t)(tj & 1) * tc_bsub_smem(1);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       sbuf + TC_ACHUNK + q * tc_bsub_smem(1)),
                   "l"(gb + (size_t)q * TC_BSUB), "r"(tc_bsub_smem(1)), "r"(mb)
                   : "memory");
  }
  st.pend[TC_B_LOAD + bf] = 1;
}

// producer: the 3xTF32 products of one K-chunk (buffer sbuf) into accumulator
// dacc (Dr at dacc, Di at dacc + 64 NB); commits to TC_B_FREE + bf, and to
// TC_B_FULL + acc after the tile's last chunk.  The descriptors of the eight
// sub-images differ from the buffer's by constant start offsets.
template <int NB>
__device__ __forceinline__ void tc_issue_mma(TcState& st, int bf, unsigned sbuf, unsigned dacc, bool first_chunk,
                                             bool last_chunk, int acc) {
  asm volatile("tcgen05.fence::after_thread_sync;");
  constexpr int TN = tc_tile_cols(NB), BS = tc_bsub_smem(NB);
  const unsigned id_pos = tc_idesc(false, TN), id_neg = tc_idesc(true, TN);
  const unsigned long long d0 = tc_desc(sbuf);  // start field: address >> 4 (buffers end below 256 KB)
  const unsigned dR = dacc, dI = dacc + TN;
#pragma unroll
  for (int ks = 0; ks < TC_KC / 8; ++ks) {
    const unsigned long long dk = d0 + (unsigned long long)((256u * ks) >> 4);
    const unsigned long long yr_hi = dk + (0 * TC_ASUB >> 4), yr_lo = dk + (1 * TC_ASUB >> 4);
    const unsigned long long yi_hi = dk + (2 * TC_ASUB >> 4), yi_lo = dk + (3 * TC_ASUB >> 4);
    const unsigned long long xr_hi = dk + ((TC_ACHUNK + 0 * BS) >> 4), xr_lo = dk + ((TC_ACHUNK + 1 * BS) >> 4);
    const unsigned long long xi_hi = dk + ((TC_ACHUNK + 2 * BS) >> 4), xi_lo = dk + ((TC_ACHUNK + 3 * BS) >> 4);
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
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   st.mb[TC_B_FREE + bf])
               : "memory");
  st.pend[TC_B_FREE + bf] = 1;
  if (last_chunk) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     st.mb[TC_B_FULL + acc])
                 : "memory");
    st.pend[TC_B_EMPTY + acc] = 1;  // the epilogue will arrive once it has read the accumulator
  }
}

// relaxed device-scope reductions W += v (16-byte aligned for the vector form);
// they are ordered before the grid barrier that ends the fold by its release fence
__device__ __forceinline__ void tc_red4(float* w, float4 v) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(w), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void tc_red1(float* w, float v) {
  asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(w), "f"(v) : "memory");
}

// 16 consecutive accumulator columns of this thread's lane (tensor-memory lane
// quadrant of the warp), as floats
__device__ __forceinline__ void tc_ld16(unsigned addr, float v[16]) {
  unsigned u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(u[q]);
}

// The tiles [t_begin, T) with step t_step, in a pipeline of three roles:
//   producer (lane 0 of warp 0): operand chunks stream through two shared
//     buffers across tile boundaries; the MMAs of a tile go to accumulator
//     k & 1 once the epilogue has read that accumulator's previous tile;
//   epilogue (the last tc_epi_warps() warps, named barrier 1): per 16-column
//     part its threads copy the accumulator rows of their lane quadrants
//     (tcgen05.ld) into a shared stage and add the stage into W_lo with
//     row-contiguous vector reductions;
//   the other warps wait at the final barrier.
// smem: tc_fold_smem(NB) bytes (operand buffers, then the stage).  Returns false
// after a timeout (the caller then calls tc_teardown with failed = true).
template <int NB>
__device__ __noinline__ bool tc_fold_tiles(const SweepArgs& a, int r, const unsigned char* imgA,
                                           const unsigned char* imgB, unsigned char* smem, TcState& st,
                                           long long t_begin, long long t_step) {
  const int n = a.n, nk = (r + TC_KC - 1) / TC_KC;
  const long long T = tc_tiles<NB>(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;
  constexpr int BUF = tc_buf_bytes(NB);
  constexpr unsigned ACC = 128u * NB;  // tensor-memory columns of one accumulator
  const int ew = tc_epi_warps(), ew0 = nwarp - ew;
  const unsigned s0 = (unsigned)__cvta_generic_to_shared(smem);
  __shared__ int s_fail, s_efail;
  if (tid == 0) s_fail = s_efail = 0;
  // earlier generic-proxy use of this shared memory before the bulk copies write it
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  const long long my_tiles = t_begin < T ? (T - 1 - t_begin) / t_step + 1 : 0;
  if (tid == 0 && my_tiles > 0) {
    // ---- producer
    bool ok = true;
    const long long total = my_tiles * nk;  // chunks of all this CTA's tiles, in order
    auto coords = [&](long long g, int& ti, int& tj, int& c) {
      const long long k = g / nk;
      c = (int)(g - k * nk);
      tc_tile<NB>(t_begin + k * t_step, n, ti, tj);
    };
    for (long long g = 0; g < total && g < TC_PREF; ++g) {  // the first chunks
      int ti, tj, c;
      coords(g, ti, tj, c);
      tc_issue_copy<NB>(st, (int)g, s0 + (unsigned)g * BUF, imgA, imgB, ti, tj, c, nk);
    }
    for (long long g = 0; g < total && ok; ++g) {
      const int bf = (int)(g % TC_NBUF);
      const long long k = g / nk;
      const int cc = (int)(g - k * nk), acc = (int)(k & 1);
      const long long gn = g + TC_PREF;
      if (gn < total) {  // copy chunk gn into its buffer once the MMAs of chunk gn - TC_NBUF are done
        const int bn = (int)(gn % TC_NBUF);
        ok = tc_wait(st, TC_B_FREE + bn);
        int ti2, tj2, c2;
        coords(gn, ti2, tj2, c2);
        if (ok) tc_issue_copy<NB>(st, bn, s0 + (unsigned)bn * BUF, imgA, imgB, ti2, tj2, c2, nk);
      }
      if (ok) ok = tc_wait(st, TC_B_LOAD + bf);
      // the epilogue has read this accumulator's previous tile (of this call or an earlier one)
      if (ok && cc == 0) ok = tc_wait(st, TC_B_EMPTY + acc);
      if (ok) tc_issue_mma<NB>(st, bf, s0 + (unsigned)bf * BUF, st.tmem + ACC * acc, cc == 0, cc == nk - 1, acc);
    }
    // no copy or MMA still reads the buffers, and every read-back arrival is
    // consumed, so that the barrier phases of the next call start in step
    for (int q = TC_B_FREE; q < TC_B_FULL && ok; ++q) ok = tc_wait(st, q);
    if (ok) ok = tc_wait(st, TC_B_EMPTY) && tc_wait(st, TC_B_EMPTY + 1);
    if (!ok) s_fail = 1;
  } else if (warp >= ew0) {
    // ---- epilogue: per part (16 columns of both planes) the warps copy
    //      their lane quadrant's accumulator rows into the stage, then all
    //      epilogue threads add the stage into W_lo with row-contiguous reductions
    const int et = tid - ew0 * 32, ethreads = ew * 32;
    const int quad = warp & 3, wpq = ew / 4, pl0 = (warp - ew0) >> 2;  // wpq = 2: one plane per warp
    const int ipt = TC_M * (TC_PC / 4) / ethreads;  // float4 items per thread and plane: 2 or 4
    float4* stage = reinterpret_cast<float4*>(smem + TC_NBUF * BUF);  // [2 planes][128 rows][4 slots]
    const unsigned lane_base = (unsigned)(32 * quad) << 16;
    bool ok = true;
    for (long long k = 0; k < my_tiles && ok; ++k) {
      int ti, tj;
      tc_tile<NB>(t_begin + k * t_step, n, ti, tj);
      const int acc = (int)(k & 1), i0 = ti * TC_M, j0 = tj * tc_tile_cols(NB);
      for (int h = 0; h < 4 * NB && ok; ++h) {  // 16-column parts of the tile
        // which of this thread's four-column items of the part lie inside W (2: all four, 1: some)
        int okv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          okv[u] = 0;
          if (u >= ipt) continue;
          const int it = et + u * ethreads, gi = i0 + (it >> 2), gj = j0 + TC_PC * h + (it & 3) * 4;
          okv[u] = gi < n ? (gj + 4 <= n ? 2 : (gj < n ? 1 : 0)) : 0;
        }
        if (h == 0) {
          // the decision to stop is taken by all epilogue threads together, so that
          // none waits at a named barrier that the others have left
          if (!tc_wait_phase(st, TC_B_FULL + acc)) s_efail = 1;
          asm volatile("tcgen05.fence::after_thread_sync;");
          asm volatile("bar.sync 1, %0;" ::"r"(ethreads) : "memory");
          if (s_efail) {
            ok = false;
            break;
          }
        }
        // accumulator rows of this warp's quadrant -> stage (Dr at column 16 h, Di 64 NB further)
        const int row = 32 * quad + lane;
        const unsigned addr = st.tmem + lane_base + ACC * acc + (unsigned)(TC_PC * h);
        for (int pl = pl0; pl < 2; pl += wpq) {
          float v[16];
          tc_ld16(addr + tc_tile_cols(NB) * pl, v);
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4)
            stage[pl * TC_M * 4 + tc_stage_slot(row, q4)] =
                make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
        }
        if (h == 4 * NB - 1) {  // this warp has read accumulator acc: one arrival per warp
          asm volatile("tcgen05.fence::before_thread_sync;");
          __syncwarp();
          if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(st.mb[TC_B_EMPTY + acc]) : "memory");
        }
        asm volatile("bar.sync 1, %0;" ::"r"(ethreads) : "memory");  // stage complete
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (!okv[u]) continue;
          const int it = et + u * ethreads, rw = it >> 2, q4 = it & 3;
          const int gi = i0 + rw, gj = j0 + TC_PC * h + 4 * q4;
          const float4 sr = stage[tc_stage_slot(rw, q4)], si = stage[TC_M * 4 + tc_stage_slot(rw, q4)];
          const size_t o = (size_t)gi * a.ldl + gj;
          // W_lo += stage as reductions performed in L2: no read on this side, so
          // the epilogue never waits for memory; one writer per element and fold,
          // one FP32 rounding per element as a load-add-store
          if (okv[u] == 2) {
            tc_red4(a.Wr + o, sr);
            tc_red4(a.Wi + o, si);
          } else {
            const float srv[4] = {sr.x, sr.y, sr.z, sr.w}, siv[4] = {si.x, si.y, si.z, si.w};
            for (int q = 0; q < 4 && gj + q < n; ++q) {
              tc_red1(a.Wr + o + q, srv[q]);
              tc_red1(a.Wi + o + q, siv[q]);
            }
          }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(ethreads) : "memory");  // stage consumed
      }
    }
    if (!ok) s_fail = 1;
  }
  __syncthreads();
  return s_fail == 0;
}

// bytes of the global operand images for a region of n pixels and r <= R delayed columns
__host__ __device__ __forceinline__ size_t tc_image_bytes(int n, int R) {
  const size_t nk = (size_t)(R + TC_KC - 1) / TC_KC;
  const size_t nI = (size_t)(n + TC_M - 1) / TC_M, nJ = (size_t)tc_njb(n);
  return nI * nk * TC_ACHUNK + nJ * nk * TC_BCHUNK;
}

}  // namespace
}  // namespace pngf
