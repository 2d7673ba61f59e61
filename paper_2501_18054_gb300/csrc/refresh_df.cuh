// Double-float refresh of the mixed search (R0 and R1 of the iterative
// refinement): x = v.[e, T] at the active pixels as FP32 pairs, and the
// residuals r = rhs - y + G x of the own rows with x2 = v.r.
#pragma once
#include "sweep_common.cuh"

namespace pngf {
namespace {

// ---------------------------------------------------------------- double-float refresh (mixed search)
// An SM of this GPU retires about 1.7 FP64 FMA lanes per clock against 128
// FP32 lanes, so the mixed search forms the residual of R1 in double-float
// arithmetic: a real number is the unevaluated sum hi + lo of two FP32 values
// (48 significant bits).
//  - product of two pairs: hi_a hi_b = p + err exactly, with p = fl(hi_a hi_b)
//    and err = fma(hi_a, hi_b, -p) (Dekker's exact product in its fused
//    multiply-add form); the cross terms hi_a lo_b + lo_a hi_b are formed in
//    FP32, lo_a lo_b (2^-48 relative) is dropped;
//  - sum: Knuth's TwoSum adds p to the running hi and keeps the rounding error
//    exactly; rounding errors and cross terms gather in lo.
// A lane's sum over k terms then errs by about k 2^-48 sum_i |G_ji x_i|, next
// to k 2^-53 for the FP64 sum and far below the FP32 drift the refresh
// removes.  Round-to-nearest intrinsics throughout keep the compiler from
// contracting a product and a sum into one FMA, which would break the exact
// transformations.
struct dfsum {  // a running sum hi + lo (the partial sums of the groups)
  float hi, lo;
};
__device__ __forceinline__ double df_value(dfsum s) { return (double)s.hi + (double)s.lo; }
// ---- packed pairs: two FP32 lanes in one 64-bit operand of the f32x2 instructions
typedef unsigned long long f2x2;
__device__ __forceinline__ f2x2 pk2(float lo, float hi) {
  f2x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(f2x2 v, float& lo, float& hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ f2x2 add2(f2x2 a, f2x2 b) {
  f2x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x2 sub2(f2x2 a, f2x2 b) {
  f2x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x2 mul2(f2x2 a, f2x2 b) {
  f2x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x2 fma2(f2x2 a, f2x2 b, f2x2 c) {
  f2x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// Two double-float multiply-adds in one instruction stream, one per lane of the
// pairs: (H, L) += (a1 + a2)(b1 + b2), with na1 = -a1 and na2 = -a2 given.
//   p = fl(a1 b1); -err = fma(-a1, b1, p) (exact); -cross = -(a1 b2 + a2 b1 + err);
//   TwoSum(H, p) = t + rnd exactly; H = t; L += rnd + cross.
// The negated operands give the error terms with the opposite sign, so no
// negation instruction is needed.
__device__ __forceinline__ void df_madd2(f2x2& H, f2x2& L, f2x2 a1, f2x2 na1, f2x2 na2, f2x2 b1, f2x2 b2) {
  const f2x2 p = mul2(a1, b1);
  const f2x2 nerr = fma2(na1, b1, p);
  const f2x2 ncross = fma2(na1, b2, fma2(na2, b1, nerr));
  const f2x2 t = add2(H, p);
  const f2x2 bv = sub2(t, H);
  const f2x2 rnd = add2(sub2(H, sub2(t, bv)), sub2(p, bv));
  H = t;
  L = add2(L, sub2(rnd, ncross));
}

// hi and lo FP32 parts of an FP64 value
__device__ __forceinline__ void df_parts(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// R0, mixed search: x = v.[e, T] at this CTA's active pixels (act, m: the
// active list in shared memory), as FP32 pairs at the pixel's rank t in the
// list, each part twice so that it is a packed operand as it stands:
// xs[2 (q n + t)] = (Re hi, Re hi, Re lo, Re lo), xs[2 (q n + t) + 1] the same of Im
template <int NV>
__device__ void refresh_x_df_t(const SweepArgs& a, int pb, int pe, const int* act, int m) {
  const int t0 = count_below(act, m, pb), t1 = count_below(act, m, pe);
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const int j = act[t];
    const c128 vj = a.v[j];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const c128 y = q == 0 ? a.e[j] : a.T[(size_t)(q - 1) * a.ldt + j];
      const c128 x = cmul(vj, y);
      float rh, rl, ih, il;
      df_parts(x.x, rh, rl);
      df_parts(x.y, ih, il);
      float4* dst = a.xs + 2 * ((size_t)q * a.n + t);
      dst[0] = make_float4(rh, rh, rl, rl);
      dst[1] = make_float4(ih, ih, il, il);
    }
  }
}

__device__ __forceinline__ void df_add(dfsum& s, float hi, float lo) {
  const float t = __fadd_rn(s.hi, hi);
  const float bv = __fsub_rn(t, s.hi);
  const float rnd = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bv)), __fsub_rn(hi, bv));
  s.hi = t;
  s.lo = __fadd_rn(s.lo, __fadd_rn(rnd, lo));
}

__device__ void refresh_x_df(const SweepArgs& a, int pb, int pe, const int* act, int m) {
  switch (a.n_o) {
    case 1: refresh_x_df_t<2>(a, pb, pe, act, m); break;
    case 2: refresh_x_df_t<3>(a, pb, pe, act, m); break;
    case 3: refresh_x_df_t<4>(a, pb, pe, act, m); break;
    case 4: refresh_x_df_t<5>(a, pb, pe, act, m); break;
    case 5: refresh_x_df_t<6>(a, pb, pe, act, m); break;
    case 6: refresh_x_df_t<7>(a, pb, pe, act, m); break;
    case 7: refresh_x_df_t<8>(a, pb, pe, act, m); break;
    default: refresh_x_df_t<9>(a, pb, pe, act, m); break;
  }
}

// R1, mixed search: residuals of own rows over the active columns in
// double-float products (G2: G as FP32 pairs), two real products per packed
// instruction stream: (Re G Re x, Im G Re x) and (-Im G Im x, Re G Im x) into
// the (Re, Im) pair of the running sum.
//
// G is symmetric, so row j at the active columns is read as the entries
// G[i][j], j in [pb, pe), of the active rows i.  Thread jl of a group of gs
// threads (own rows rounded up to a warp) takes own row pb + jl (lanes past
// the own rows repeat the last one); the ng = blockDim / gs groups take the
// active list in turn.  A stage is S = ng R consecutive list entries, R per
// group, and the operands travel by asynchronous 16-byte copies into a ring
// of RD_D stages: every thread copies the G entries it multiplies itself, and
// every warp the x entries of its group's rows (x: NV x R x 2 float4 per warp
// and stage).  A thread therefore waits only for its own copies (cp.async groups,
// one per stage) and a warp-level barrier, and the warps run through the
// ring independently, RD_D - 1 stages in flight.
//
// The groups' partial sums are then added in shared memory, one vector at a
// time and in group order, and r and x2 = v.r are formed in FP64.
//
// area, area_bytes: 16-byte aligned shared memory for the ring (the partial
// sums reuse it: blockDim float4).
constexpr int RD_D = 3;
constexpr float kRefreshGuard = 1e-3f;  // largest relative residual of e the mixed search accepts
constexpr int RD_RMAX = 8;
// list entries per group and stage for own rows and NV vectors in area_bytes (0: too small)
__host__ __device__ __forceinline__ int rd_rows(int own, int NV, int nthreads, unsigned area_bytes) {
  const int gs = (own + 31) & ~31, ng = nthreads / gs;
  const unsigned per_r = (unsigned)(ng * gs) * 16u + (unsigned)(nthreads / 32) * (unsigned)NV * 32u;
  const int R = (int)(area_bytes / ((unsigned)RD_D * per_r));
  return R < RD_RMAX ? R : RD_RMAX;
}

template <int NV>
__device__ __noinline__ void refresh_residual_df_t(const SweepArgs& a, int pb, int pe, const int* act, int m,
                                                   unsigned char* area, unsigned area_bytes) {
  const int own = pe - pb, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)blockDim.x >> 5;
  const int gs = (own + 31) & ~31, ng = (int)blockDim.x / gs;  // own <= blockDim
  const int grp = tid / gs, jl = tid - grp * gs, jc = min(jl, own - 1);
  const int R = rd_rows(own, NV, (int)blockDim.x, area_bytes);  // >= 1: checked by the host
  const int S = ng * R;
  // a stage: G entries [ng R][gs] float4 (group g's rows at g R), then x [nw][NV][R][2] float4
  const unsigned stage = (unsigned)(S * gs) * 16u + (unsigned)(nw * NV * R) * 32u;
  const unsigned oX = (unsigned)(S * gs) * 16u;
  const int nst = (m + S - 1) / S;
  const unsigned s0 = (unsigned)__cvta_generic_to_shared(area);
  const bool live = grp < ng;
  // this lane's x copies: the same slots and source offsets every stage, the list position
  // moving by S (x_t: position within a stage, -1 = none)
  constexpr int XMAX = (2 * 9 * RD_RMAX + 31) / 32;
  int x_t[XMAX];
  unsigned x_dst[XMAX];
  size_t x_src[XMAX];
#pragma unroll
  for (int u = 0; u < XMAX; ++u) {
    const int e = lane + 32 * u;
    x_t[u] = -1;
    x_dst[u] = 0;
    x_src[u] = 0;
    if (e < 2 * NV * R) {
      const int h = e & 1, qr = e >> 1, q = qr / R, r = qr - q * R;
      x_t[u] = grp + ng * r;
      x_dst[u] = oX + (unsigned)(((warp * NV + q) * R + r) * 2 + h) * 16u;
      x_src[u] = 2 * (size_t)q * a.n + h;
    }
  }
  // this thread's copies of stage k into slot k % RD_D (always one cp.async group)
  auto issue = [&](int k) {
    if (live && k < nst) {
      const unsigned dst = s0 + (unsigned)(k % RD_D) * stage;
      for (int r = 0; r < R; ++r) {
        const int t = k * S + grp + ng * r;
        if (t >= m) break;
        const float4* src = a.G2 + (size_t)act[t] * a.n + pb + jc;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + (unsigned)((grp * R + r) * gs + jl) * 16u),
                     "l"(src)
                     : "memory");
      }
#pragma unroll
      for (int u = 0; u < XMAX; ++u) {
        const int t = k * S + x_t[u];
        if (x_t[u] >= 0 && t < m)
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + x_dst[u]), "l"(a.xs + x_src[u] + 2 * t)
                       : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // earlier use of this shared memory (the active list's neighbours, the delayed set) is complete
  __syncthreads();
  for (int k = 0; k < RD_D - 1; ++k) issue(k);
  f2x2 H[NV], L[NV];  // (Re, Im) of the running sums: hi parts, lo parts
#pragma unroll
  for (int q = 0; q < NV; ++q) H[q] = L[q] = 0ull;
  for (int k = 0; k < nst; ++k) {
    __syncwarp();  // this warp is done with slot (k - 1) % RD_D, which stage k + RD_D - 1 refills
    issue(k + RD_D - 1);
    asm volatile("cp.async.wait_group %0;" ::"n"(RD_D - 1) : "memory");  // stage k has landed
    __syncwarp();                                                         // ... for every lane of the warp
    if (!live) continue;
    const unsigned char* st = area + (size_t)(k % RD_D) * stage;
    const ulonglong2* gst = reinterpret_cast<const ulonglong2*>(st) + grp * R * gs + jl;
    const ulonglong2* xst = reinterpret_cast<const ulonglong2*>(st + oX) + warp * NV * R * 2;
    const int tk = k * S + grp, rc = tk < m ? min(R, (m - tk + ng - 1) / ng) : 0;
    for (int r = 0; r < rc; ++r) {
      const ulonglong2 g = gst[r * gs];  // (Re hi, Im hi), (Re lo, Im lo) of G
      float gr1, gi1, gr2, gi2;
      upk2(g.x, gr1, gi1);
      upk2(g.y, gr2, gi2);
      const f2x2 na1 = pk2(-gr1, -gi1), na2 = pk2(-gr2, -gi2);
      const f2x2 b1 = pk2(-gi1, gr1), nb1 = pk2(gi1, -gr1), nb2 = pk2(gi2, -gr2);
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const ulonglong2 xr = xst[(q * R + r) * 2], xi = xst[(q * R + r) * 2 + 1];
        df_madd2(H[q], L[q], g.x, na1, na2, xr.x, xr.y);  // (Re G Re x, Im G Re x)
        df_madd2(H[q], L[q], b1, nb1, nb2, xi.x, xi.y);   // (-Im G Im x, Re G Im x)
      }
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __shared__ unsigned s_rmax, s_ymax;  // non-negative FP32 magnitudes as ordered bit patterns
  if (tid == 0) s_rmax = s_ymax = 0u;
  __syncthreads();
  float4* part = reinterpret_cast<float4*>(area);
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    if (live) {
      float rh, ih, rl, il;
      upk2(H[q], rh, ih);
      upk2(L[q], rl, il);
      part[tid] = make_float4(rh, rl, ih, il);
    }
    __syncthreads();
    if (tid < own) {
      dfsum re{0.f, 0.f}, im{0.f, 0.f};
      for (int g2 = 0; g2 < ng; ++g2) {
        const float4 p = part[g2 * gs + tid];
        df_add(re, p.x, p.y);
        df_add(im, p.z, p.w);
      }
      const int j = pb + tid;
      const c128 rhs = q == 0 ? a.cd[j] : a.God[(size_t)(q - 1) * a.n + j];
      const c128 y = q == 0 ? a.e[j] : a.T[(size_t)(q - 1) * a.ldt + j];
      const c128 r = cadd(csub(rhs, y), mk(df_value(re), df_value(im)));
      rvec(a, 0, q)[j] = r;
      if (q == 0) {  // accuracy guard on the field's residual
        atomicMax(&s_rmax, __float_as_uint((float)cabs1(r)));
        atomicMax(&s_ymax, __float_as_uint((float)cabs1(y)));
      }
      const c128 x2 = cmul(a.v[j], r);
      x2f(a, q)[j] = make_float2((float)x2.x, (float)x2.y);
    }
    __syncthreads();
  }
  // The refresh corrects e and T by one refinement step with the FP32 inverse,
  // which converges only while |r| stays far below |e|: between refreshes the
  // FP32 drift leaves |r| ~ 1e-7 |e| on well-conditioned systems.  A residual
  // above kRefreshGuard |e| (an ill-conditioned system, e.g. a design driven
  // into a high-Q resonance) means the maintained state has lost accuracy.
  if (tid == 0 && __uint_as_float(s_rmax) > kRefreshGuard * __uint_as_float(s_ymax))
    latch_status(a.ctl, PNGF_EACCURACY);
}

__device__ void refresh_residual_df(const SweepArgs& a, int pb, int pe, const int* act, int m, unsigned char* area,
                                    unsigned area_bytes) {
  switch (a.n_o) {
    case 1: refresh_residual_df_t<2>(a, pb, pe, act, m, area, area_bytes); break;
    case 2: refresh_residual_df_t<3>(a, pb, pe, act, m, area, area_bytes); break;
    case 3: refresh_residual_df_t<4>(a, pb, pe, act, m, area, area_bytes); break;
    case 4: refresh_residual_df_t<5>(a, pb, pe, act, m, area, area_bytes); break;
    case 5: refresh_residual_df_t<6>(a, pb, pe, act, m, area, area_bytes); break;
    case 6: refresh_residual_df_t<7>(a, pb, pe, act, m, area, area_bytes); break;
    case 7: refresh_residual_df_t<8>(a, pb, pe, act, m, area, area_bytes); break;
    default: refresh_residual_df_t<9>(a, pb, pe, act, m, area, area_bytes); break;
  }
}

// ---------------------------------------------------------------- FP32 correction, balanced (mixed search)
// y = W x2 for every row (W symmetric, its upper triangle current in the FP32
// planes, x2 = v.r), with the triangle's work dealt evenly over the grid
// instead of by own rows (own rows near the top of the triangle carry the
// longest rows, so the CTA holding them set the pace of the whole refresh):
//  - upper part sum_{i>=j} W[j][i] x2_i, row by row in groups of 2 nw rows: a
//    warp takes rows j and j + nw, which share every staged x2 read, lanes read
//    four-wide along the rows;
//  - lower part sum_{i<j} W[i][j] x2_i, column by column in blocks of 32
//    (lane = column), over the active rows i < j only (x2 vanishes elsewhere).
// Round k of the groups (of the blocks) gives CTA c item k G + c for even k and
// k G + G - 1 - c for odd k: the snake pairs long rows with short ones and
// tall column blocks with low ones.  Upper sums go to block 3 of the scratch,
// lower sums to block 1; correct_combine adds r + upper + lower into e and T of
// the own rows once a grid barrier has made them visible.
// act: the ascending active-pixel list (global memory), m its length; smem:
// smem_bytes of shared memory (16-byte aligned).
__device__ __forceinline__ int snake_item(int k, int c, int G) { return k * G + ((k & 1) ? G - 1 - c : c); }

template <int NV>
__device__ __noinline__ void correct_balanced_t(const SweepArgs& a, const int* act, int m, float* smem, int smem_bytes) {
  const int n = a.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)blockDim.x >> 5;
  const int G = (int)gridDim.x, cta = (int)blockIdx.x;
  float2* red = reinterpret_cast<float2*>(smem);  // [warps][NV][32]
  float2* xs = red + nw * NV * 32;
  const int avail = smem_bytes - nw * NV * 32 * (int)sizeof(float2);
  // ---- upper part
  const int n128 = (n + 127) & ~127;
  const int cw = min(n128, avail / (NV * (int)sizeof(float2)) / 128 * 128);
  const bool whole = cw >= n128;  // x2 staged once for every group
  const int RG = 2 * nw, n_groups = (n + RG - 1) / RG;
  bool staged = false;
  for (int k = 0; k * G < n_groups; ++k) {
    const int g = snake_item(k, cta, G);
    if (g >= n_groups) continue;
    const int g0 = g * RG, j1 = g0 + warp, j2 = g0 + warp + nw;
    f2c acc1[NV], acc2[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc1[q] = acc2[q] = f2c{0.f, 0.f};
    const int cstart = whole ? 0 : (g0 & ~127);
    for (int c0 = cstart; c0 < n; c0 += cw) {
      if (!whole || !staged) {
        __syncthreads();
        // column cc of the chunk at (cc & 3) * (cw / 4) + (cc >> 2): lanes read consecutive words;
        // four reads in flight per thread before their stores
        for (int e0 = tid; e0 < NV * cw; e0 += 4 * blockDim.x) {
          float2 v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x, q = e / cw, cc = e - q * cw, col = c0 + cc;
            v[u] = e < NV * cw && col < n ? x2f(a, q)[col] : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x, q = e / cw, cc = e - q * cw;
            if (e < NV * cw) xs[q * cw + (cc & 3) * (cw >> 2) + (cc >> 2)] = v[u];
          }
        }
        __syncthreads();
        staged = true;
      }
      if (j1 < n) {
        const int kb = max(0, ((j1 & ~3) - c0) >> 7), ke = min(cw, n - c0 + 127) >> 7;
        for (int k0 = kb; k0 < ke; k0 += 4) {  // four four-wide reads of each row in flight per lane
          f2c w1[4][4], w2[4][4];
#pragma unroll
          for (int u4 = 0; u4 < 4; ++u4) {
            const int col = c0 + 128 * (k0 + u4) + 4 * lane;
            const bool in = k0 + u4 < ke && col < n;
            if (in && col + 3 >= j1) {
              w_row4<true>(a, j1, col, w1[u4]);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) w1[u4][u] = f2c{0.f, 0.f};
            }
            if (in && j2 < n && col + 3 >= j2) {
              w_row4<true>(a, j2, col, w2[u4]);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) w2[u4][u] = f2c{0.f, 0.f};
            }
          }
#pragma unroll
          for (int u4 = 0; u4 < 4; ++u4) {
            const int kk = k0 + u4;
            if (kk < ke) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int i = c0 + 128 * kk + 4 * lane + u;
                const bool ok1 = i >= j1 && i < n, ok2 = i >= j2 && i < n;
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                  const float2 x = xs[q * cw + u * (cw >> 2) + 32 * kk + lane];
                  if (ok1) acc1[q] = f2fma(w1[u4][u], f2c{x.x, x.y}, acc1[q]);
                  if (ok2) acc2[q] = f2fma(w2[u4][u], f2c{x.x, x.y}, acc2[q]);
                }
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const f2c s1 = f2sum(acc1[q]), s2 = f2sum(acc2[q]);
      if (lane == 0 && j1 < n) rvec(a, 3, q)[j1] = mk(s1.x, s1.y);
      if (lane == 0 && j2 < n) rvec(a, 3, q)[j2] = mk(s2.x, s2.y);
    }
  }
  // ---- lower part: blocks of 32 columns, rows from the staged active list
  const int rcap = max(1, min(max(m, 1), avail / (int)(sizeof(int) + NV * sizeof(float2))));
  int* rows = reinterpret_cast<int*>(xs + NV * rcap);
  const bool fits = m <= rcap;  // every active row staged once
  if (fits) {
    __syncthreads();
    for (int e = tid; e < m; e += blockDim.x) rows[e] = act[e];
    __syncthreads();
    for (int e0 = tid; e0 < NV * m; e0 += 4 * blockDim.x) {  // four reads in flight per thread
      float2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * blockDim.x, q = e / m, tt = e - q * m;
        v[u] = e < NV * m ? x2f(a, q)[rows[tt]] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * blockDim.x, q = e / m, tt = e - q * m;
        if (e < NV * m) xs[q * rcap + tt] = v[u];
      }
    }
    __syncthreads();
  }
  const int n_blocks = (n + 31) / 32;
  for (int k = 0; k * G < n_blocks; ++k) {
    const int bi = snake_item(k, cta, G);
    if (bi >= n_blocks) continue;
    const int cb = bi * 32, j = cb + lane;
    const bool colok = j < n;
    // active rows above the block's last column (searched in the staged copy when it holds them all)
    const int t_blk = count_below(fits ? rows : act, m, min(cb + 31, n - 1));
    f2c acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = f2c{0.f, 0.f};
    for (int t0 = 0; t0 < t_blk; t0 += rcap) {
      const int cnt = min(rcap, t_blk - t0);
      if (!fits) {
        __syncthreads();
        for (int e = tid; e < cnt; e += blockDim.x) rows[e] = act[t0 + e];
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
            if (colok && i < j) w[u] = w_upper<true>(a, i, j);
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
    // the warps' column partials, summed in warp order
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
      rvec(a, 1, q)[j] = mk((double)sx, (double)sy);
    }
    __syncthreads();
  }
}

__device__ void correct_balanced(const SweepArgs& a, const int* act, int m, float* smem, int smem_bytes) {
  switch (a.n_o) {
    case 1: correct_balanced_t<2>(a, act, m, smem, smem_bytes); break;
    case 2: correct_balanced_t<3>(a, act, m, smem, smem_bytes); break;
    case 3: correct_balanced_t<4>(a, act, m, smem, smem_bytes); break;
    case 4: correct_balanced_t<5>(a, act, m, smem, smem_bytes); break;
    case 5: correct_balanced_t<6>(a, act, m, smem, smem_bytes); break;
    case 6: correct_balanced_t<7>(a, act, m, smem, smem_bytes); break;
    case 7: correct_balanced_t<8>(a, act, m, smem, smem_bytes); break;
    default: correct_balanced_t<9>(a, act, m, smem, smem_bytes); break;
  }
}

// e, T of the own rows += r + upper + lower (after the grid barrier that
// follows correct_balanced)
__device__ void correct_combine(const SweepArgs& a, int pb, int pe) {
  const int own = pe - pb, nv = 1 + a.n_o;
  for (int e = threadIdx.x; e < nv * own; e += blockDim.x) {
    const int q = e / own, j = pb + (e - q * own);
    const c128 d = cadd(rvec(a, 0, q)[j], cadd(rvec(a, 3, q)[j], rvec(a, 1, q)[j]));
    c128* dst = q == 0 ? a.e + j : a.T + (size_t)(q - 1) * a.ldt + j;
    *dst = cadd(*dst, d);
  }
}

}  // namespace
}  // namespace pngf
