// Direct binary search over tile flips on one or several systems that share
// the design (FP64).
//
// A candidate flips every pixel of one tile at once: the paper's rank-M flips
// (section "Low-rank update evaluation": dP = Q^T H_P Q with M nonzero
// entries, the Woodbury update of Eq. 9 and the direct port evaluation of
// Eq. 14; its designs flip 2 to 4 symmetry-tied tiles of 24 unknowns each,
// Methods, "Optimization parameters").  Several systems -- one per frequency
// in the paper ("Computational efficiency": one G, G_obj and C^-1 per
// frequency, independent and updated side by side) -- are advanced on one
// design, and their objectives are combined into one scalar by a mean or a
// min-max rule (Supplementary Note 9).
//
// Field form (Supplementary Note 4; W = M^-1 G complex symmetric, T = G_od
// (I + V W)) for a tile K of m pixels with contrast changes D = diag(delta_K):
//   A = I - D W_KK (the m x m capacitance matrix), y = A^-1 D e_K,
//   o(new) = o + T[:, K] y                                       (score)
//   Z = A^-1 D (complex symmetric), U = W[:, K], V = U Z,
//   W += V U^T, e += U y, T += (T[:, K] Z) U^T, diag W += rowdot(V, U) (accept)
// For m = 1 these are the rank-1 formulas of the single-pixel kernels.
//
// One cooperative launch runs the search.  Each CTA owns a contiguous chunk
// of tiles (scored one warp per tile and system, the m x m system solved by
// Gauss-Jordan elimination with partial pivoting, one lane per row), a
// contiguous chunk of pixels (state update) and an equal range of the packed
// upper triangle of every system's W (rank-m update).  Three grid barriers
// per kept flip: after the selection, after the gather of U and V, after the
// update (the next scores read W_KK, e_K and T[:, K] of any CTA's pixels).
#include <cstdio>

#include "sweep_common.cuh"

namespace pngf {
namespace {

constexpr int kMaxSys = PNGF_TILES_MAX_SYSTEMS;
constexpr int kTileMax = PNGF_TILE_MAX;
constexpr int kWarps = kThreads / 32;
constexpr int kScoreCols = kTileMax + 1;        // [A | rhs]
constexpr int kScoreLd = kScoreCols + 1;        // padded row stride (complex entries)
constexpr int kAcceptLd = 2 * kTileMax + 1;     // [A | D], padded

struct GenArgs {
  SweepArgs sys[kMaxSys];
  int n_sys, combine, kind;
  const int* tiles;  // n_tiles x tile_m, -1 pads
  int n_tiles, tile_m;
  c128* U;  // [n_sys][n][tile_m]
  c128* V;  // [n_sys][n][tile_m]
  int* pos_of;  // n_tiles
  double* part_gain;  // [2][P]
  long long* part_key;
  int mode, n_sweeps, trace_cap, refresh_k, forced_tile;
  const int* order;  // n_sweeps x n_tiles
  int32_t* trace;
  double* trace_f;
  int64_t* counters;
  double tau;
};

__device__ __forceinline__ c128 w_sym(const SweepArgs& a, int i, int j) {
  return i <= j ? a.W[(size_t)i * a.ldw + j] : a.W[(size_t)j * a.ldw + i];
}

__device__ __forceinline__ double combine_of(const double* f, int n_sys, int combine, int kind) {
  double r = f[0];
  if (combine == PNGF_COMBINE_MEAN) {
    for (int s = 1; s < n_sys; ++s) r += f[s];
    return r / n_sys;
  }
  for (int s = 1; s < n_sys; ++s) r = kind == PNGF_OBJ_MAX_WEIGHTED_POWER ? fmin(r, f[s]) : fmax(r, f[s]);
  return r;
}

// the tile's pixels, compacted: lane i < m gets the i-th valid pixel; invalid
// entries (outside [-1, n)) make the tile unusable (bad = true on every lane)
__device__ __forceinline__ int tile_pixels(const GenArgs& g, int t, int n, int& m, bool& bad) {
  const int lane = threadIdx.x & 31;
  int px = lane < g.tile_m ? g.tiles[(size_t)t * g.tile_m + lane] : -1;
  bad = __any_sync(0xffffffffu, px < -1 || px >= n);
  const unsigned valid = __ballot_sync(0xffffffffu, px >= 0);
  m = __popc(valid);
  // lane i fetches the i-th valid pixel
  int mine = -1;
  for (int src = 0; src < g.tile_m; ++src) {
    const int v = __shfl_sync(0xffffffffu, px, src);
    const int s = __popc(valid & ((1u << src) - 1u));
    if (((valid >> src) & 1u) && s == lane) mine = v;
  }
  return mine;
}

// Gauss-Jordan elimination with partial pivoting on the m x ncols system held
// in shared memory (row r at A + r * ld), one lane per row; on success the
// first m columns are the identity and the rest hold A^-1 [rhs].  A pivot
// below 1e-14 in magnitude marks the candidate singular (the single-pixel
// paths skip |d_k| < 1e-14 the same way).  Warp-uniform result.
__device__ bool warp_gauss_jordan(c128* A, int ld, int m, int ncols) {
  const int lane = threadIdx.x & 31;
  for (int c = 0; c < m; ++c) {
    double mag = (lane >= c && lane < m) ? cabs2(A[lane * ld + c]) : -1.0;
    int piv = lane;
    for (int off = 16; off > 0; off >>= 1) {
      const double om = __shfl_xor_sync(0xffffffffu, mag, off);
      const int op = __shfl_xor_sync(0xffffffffu, piv, off);
      if (om > mag || (om == mag && op < piv)) { mag = om; piv = op; }
    }
    if (!(mag >= 1e-28)) return false;
    if (piv != c)
      for (int j = lane; j < ncols; j += 32) {
        const c128 t = A[c * ld + j];
        A[c * ld + j] = A[piv * ld + j];
        A[piv * ld + j] = t;
      }
    __syncwarp();
    const c128 inv = cdiv(mk(1.0, 0.0), A[c * ld + c]);
    __syncwarp();
    for (int j = lane; j < ncols; j += 32) A[c * ld + j] = j == c ? mk(1.0, 0.0) : cmul(A[c * ld + j], inv);
    __syncwarp();
    if (lane < m && lane != c) {
      const c128 l = A[lane * ld + c];
      for (int j = c; j < ncols; ++j) A[lane * ld + j] = j == c ? mk(0.0, 0.0) : cfms(l, A[c * ld + j], A[lane * ld + j]);
    }
    __syncwarp();
  }
  return true;
}

// contrast change of pixel k if flipped: +dv (off -> on) or -dv (on -> off)
__device__ __forceinline__ c128 delta_of(const SweepArgs& a, int k) {
  const c128 d = a.dv[k];
  return a.b[k] ? mk(-d.x, -d.y) : d;
}

// Score one tile in one system (one warp): f after the flip, or false if the
// capacitance system is singular.  o: the system's current ports; buf: the
// warp's kTileMax x kScoreLd scratch.
__device__ bool score_tile_sys(const SweepArgs& a, const ObjParams& op, const c128* o, int px, int m, c128* buf,
                               double& f_new, c128* o_new) {
  const int lane = threadIdx.x & 31;
  // row `lane` of [I - D W_KK | D e_K]
  if (lane < m) {
    const c128 dl = delta_of(a, px);
    for (int j = 0; j < m; ++j) {
      const int pj = __shfl_sync((1u << m) - 1u, px, j);
      const c128 w = w_sym(a, px, pj);
      const c128 dw = cmul(dl, w);
      buf[lane * kScoreLd + j] = j == lane ? csub(mk(1.0, 0.0), dw) : mk(-dw.x, -dw.y);
    }
    buf[lane * kScoreLd + m] = cmul(dl, a.e[px]);
  }
  __syncwarp();
  if (!warp_gauss_jordan(buf, kScoreLd, m, m + 1)) return false;
  const c128 y = lane < m ? buf[lane * kScoreLd + m] : mk(0.0, 0.0);
  double f = 0.0;
#pragma unroll 1
  for (int p = 0; p < a.n_o; ++p) {
    c128 t = lane < m ? cmul(a.T[(size_t)p * a.ldt + px], y) : mk(0.0, 0.0);
    t = warp_sum(t);  // every lane holds the sum
    const c128 on = cadd(o[p], t);
    if (o_new) o_new[p] = on;
    f += objective_term(op, p, on);
  }
  f_new = f;
  __syncwarp();
  return true;
}

// Single-pixel tiles (tile_m = 1), one thread per candidate: the same
// arithmetic as the warp path for m = 1 (pivot 1 - delta W_kk, its reciprocal,
// then (delta e_k) times it), so both paths take the same decisions.
__device__ bool score_pixel_tile(const GenArgs& g, const c128 (*s_o)[kMaxPorts], int t, double& F) {
  const int k = g.tiles[t];
  if (k < -1 || k >= g.sys[0].n) {
    latch_status(g.sys[0].ctl, PNGF_EINVAL);
    return false;
  }
  if (k < 0) return false;
  double fs[kMaxSys];
  for (int s = 0; s < g.n_sys; ++s) {
    const SweepArgs& a = g.sys[s];
    const c128 dl = delta_of(a, k);
    const c128 A = csub(mk(1.0, 0.0), cmul(dl, a.diag[k]));
    if (!(cabs2(A) >= 1e-28)) return false;
    const c128 y = cmul(cmul(dl, a.e[k]), cdiv(mk(1.0, 0.0), A));
    double f = 0.0;
#pragma unroll 1
    for (int p = 0; p < a.n_o; ++p) f += objective_term(a.op, p, cadd(s_o[s][p], cmul(a.T[(size_t)p * a.ldt + k], y)));
    fs[s] = f;
  }
  F = combine_of(fs, g.n_sys, g.combine, g.kind);
  return true;
}

// combined objective of flipping tile t (one warp); false if any system is singular
__device__ bool score_tile(const GenArgs& g, const c128 (*s_o)[kMaxPorts], int t, c128* buf, double& F,
                           double* f_sys) {
  int m;
  bool bad;
  const int px = tile_pixels(g, t, g.sys[0].n, m, bad);
  if (bad && (threadIdx.x & 31) == 0) latch_status(g.sys[0].ctl, PNGF_EINVAL);
  if (bad || m == 0) return false;
  double fs[kMaxSys];
  for (int s = 0; s < g.n_sys; ++s) {
    if (!score_tile_sys(g.sys[s], g.sys[s].op, s_o[s], px, m, buf, fs[s], nullptr)) return false;
    if (f_sys) f_sys[s] = fs[s];
  }
  F = combine_of(fs, g.n_sys, g.combine, g.kind);
  return true;
}

// Pivot of a kept tile in one system (warp 0 of every CTA, identical results):
// Z = (I - D W_KK)^-1 D into z (m x m, row-major), y = Z e_K, tz = T[:, K] Z
// (n_o x m), o += T[:, K] y.  buf: kTileMax x kAcceptLd scratch.
__device__ bool accept_pivot_sys(const SweepArgs& a, int px, int m, c128* buf, c128* z, c128* y, c128* tz, c128* o) {
  const int lane = threadIdx.x & 31;
  c128 dl = mk(0.0, 0.0);
  if (lane < m) {
    dl = delta_of(a, px);
    for (int j = 0; j < m; ++j) {
      const int pj = __shfl_sync((1u << m) - 1u, px, j);
      const c128 dw = cmul(dl, w_sym(a, px, pj));
      buf[lane * kAcceptLd + j] = j == lane ? csub(mk(1.0, 0.0), dw) : mk(-dw.x, -dw.y);
      buf[lane * kAcceptLd + m + j] = j == lane ? dl : mk(0.0, 0.0);
    }
  }
  __syncwarp();
  if (!warp_gauss_jordan(buf, kAcceptLd, m, 2 * m)) return false;
  if (lane < m)
    for (int j = 0; j < m; ++j) z[lane * kTileMax + j] = buf[lane * kAcceptLd + m + j];
  __syncwarp();
  // y_i = sum_j Z_ij e_Kj (lane i)
  const c128 ek = lane < m ? a.e[px] : mk(0.0, 0.0);
  c128 yi = mk(0.0, 0.0);
  for (int j = 0; j < m; ++j) {
    const c128 ej = mk(__shfl_sync(0xffffffffu, ek.x, j), __shfl_sync(0xffffffffu, ek.y, j));
    if (lane < m) yi = cfma(z[lane * kTileMax + j], ej, yi);
  }
  if (lane < m) y[lane] = yi;
  // tz[p][a] = sum_b T[p][K_b] Z[b][a] (lane a); o_p += sum_b T[p][K_b] y_b
#pragma unroll 1
  for (int p = 0; p < a.n_o; ++p) {
    const c128 tk = lane < m ? a.T[(size_t)p * a.ldt + px] : mk(0.0, 0.0);
    c128 acc = mk(0.0, 0.0);
    for (int b = 0; b < m; ++b) {
      const c128 tb = mk(__shfl_sync(0xffffffffu, tk.x, b), __shfl_sync(0xffffffffu, tk.y, b));
      if (lane < m) acc = cfma(tb, z[b * kTileMax + lane], acc);
    }
    if (lane < m) tz[p * kTileMax + lane] = acc;
    const c128 t = warp_sum(lane < m ? cmul(tk, yi) : mk(0.0, 0.0));
    if (lane == 0) o[p] = cadd(o[p], t);
  }
  __syncwarp();
  return true;
}

__global__ void __launch_bounds__(kThreads) dbs_tiles_kernel(const __grid_constant__ GenArgs g) {
  extern __shared__ __align__(16) unsigned char gen_smem[];
  const int P = gridDim.x, cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = g.sys[0].n, nt = g.n_tiles, M = g.tile_m;
  const int pb = (int)((long long)n * cta / P), pe = (int)((long long)n * (cta + 1) / P);
  const int tb = (int)((long long)nt * cta / P), te = (int)((long long)nt * (cta + 1) / P);
  const long long E = (long long)n * (n + 1) / 2;
  const long long eb = E * cta / P, ee = E * (cta + 1) / P;
  Control* ctl = g.sys[0].ctl;
  hold_if_asked(ctl);
  __shared__ c128 s_o[kMaxSys][kMaxPorts], s_o_new[kMaxSys][kMaxPorts];
  __shared__ double s_f[kMaxSys], s_f_new[kMaxSys];
  __shared__ double s_F;
  __shared__ c128 s_z[kMaxSys][kTileMax * kTileMax];
  __shared__ c128 s_y[kMaxSys][kTileMax];
  __shared__ c128 s_tz[kMaxSys][kMaxPorts * kTileMax];
  __shared__ int s_px[kTileMax];
  __shared__ int s_m, s_k, s_pos, s_bad;
  __shared__ c128 s_acc_buf[kTileMax * kAcceptLd];
  c128* wbuf = reinterpret_cast<c128*>(gen_smem) + (size_t)warp * kTileMax * kScoreLd;
  if (tid == 0) {
    for (int s = 0; s < g.n_sys; ++s) {
      FOR_PORTS(p, g.sys[s].n_o) s_o[s][p] = g.sys[s].ctl->o[p];
      s_f[s] = g.sys[s].ctl->f;
    }
    s_F = combine_of(s_f, g.n_sys, g.combine, g.kind);
  }
  __syncthreads();
  long long n_acc = 0, n_evals = 0, n_refresh = 0, sum_active = 0;
  int sweeps_done = 0, converged = 0, status = PNGF_OK;
  int since_refresh = g.sys[0].ctl->since_refresh;
  int s = 0, t = 0, acc_in_sweep = 0, slot = 0, rd = 0;
  bool failed = false;
  auto setup_sweep = [&](int sw) {
    if (g.order)
      for (int q = tb + tid; q < te; q += blockDim.x) {
        const int ti = g.order[(size_t)sw * nt + q];
        if ((unsigned)ti < (unsigned)nt) g.pos_of[ti] = q;
        else latch_status(ctl, PNGF_EINVAL);
      }
  };
  const bool forced = g.forced_tile >= 0;
  if (!forced && g.mode == PNGF_FIRST_IMPROVEMENT && g.order) {
    setup_sweep(0);
    if (!grid_sync(ctl)) failed = true;
    else if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) status = PNGF_EINVAL;
  }
  while (!failed && status != PNGF_EINVAL) {
    const double F = s_F;
    const double thr = g.tau * fmax(fabs(F), 1e-30);
    // ---- score this CTA's tiles (one warp per tile), reduce to the CTA's candidate
    if (!forced) {
      const bool px1 = M == 1;  // single-pixel tiles: one thread per candidate
      const int t0 = px1 ? tid : warp, ts = px1 ? (int)blockDim.x : kWarps;
      if (g.mode == PNGF_FIRST_IMPROVEMENT) {
        long long best = LLONG_MAX;
        for (int ti = tb + t0; ti < te; ti += ts) {
          const int pos = g.order ? g.pos_of[ti] : ti;
          if (pos < t || pos >= best) continue;
          double Fn;
          if (!(px1 ? score_pixel_tile(g, s_o, ti, Fn) : score_tile(g, s_o, ti, wbuf, Fn, nullptr))) continue;
          const double gain = g.kind == PNGF_OBJ_MAX_WEIGHTED_POWER ? Fn - F : F - Fn;
          if (gain - thr > 0.0) best = pos;
        }
        best = block_min_ll(px1 || lane == 0 ? best : LLONG_MAX);
        if (tid == 0) sel_offer(ctl, rd, best, cta);
      } else {
        double gb = -INFINITY;
        int pix = INT_MAX;
        for (int ti = tb + t0; ti < te; ti += ts) {
          double Fn;
          if (!(px1 ? score_pixel_tile(g, s_o, ti, Fn) : score_tile(g, s_o, ti, wbuf, Fn, nullptr))) continue;
          const double gain = g.kind == PNGF_OBJ_MAX_WEIGHTED_POWER ? Fn - F : F - Fn;
          if (better(gain, ti, gb, pix)) { gb = gain; pix = ti; }
        }
        if (!px1 && lane != 0) { gb = -INFINITY; pix = INT_MAX; }
        block_best(gb, pix);
        if (tid == 0) {
          g.part_gain[slot * P + cta] = gb;
          g.part_key[slot * P + cta] = pix;
        }
      }
      if (!grid_sync(ctl)) { failed = true; break; }
    }
    // ---- the kept tile (every CTA derives the same), its pivot in every system
    if (warp == 0) {
      int k = -1, pos_k = -1;
      if (forced) {
        k = g.forced_tile < nt ? g.forced_tile : -2;
        pos_k = 0;
      } else if (g.mode == PNGF_FIRST_IMPROVEMENT) {
        const unsigned long long key = sel_read(ctl, rd);
        if (key != ~0ull) {
          pos_k = (int)(key >> 10);
          k = g.order ? g.order[(size_t)s * nt + pos_k] : pos_k;
          if ((unsigned)k >= (unsigned)nt) k = -2;
        }
      } else {
        double gb = -INFINITY;
        int pix = INT_MAX;
        for (int q = lane; q < P; q += 32) {
          const double gg = g.part_gain[slot * P + q];
          const int pp = (int)g.part_key[slot * P + q];
          if (better(gg, pp, gb, pix)) { gb = gg; pix = pp; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const double og = __shfl_xor_sync(0xffffffffu, gb, off);
          const int op = __shfl_xor_sync(0xffffffffu, pix, off);
          if (better(og, op, gb, pix)) { gb = og; pix = op; }
        }
        if (pix != INT_MAX && gb - thr > 0.0) k = pix;
        pos_k = 0;
      }
      int bad = 0;
      if (k >= 0) {
        int m;
        bool badt;
        const int px = tile_pixels(g, k, n, m, badt);
        if (badt || m == 0) {
          bad = 1;
        } else {
          if (lane < m) s_px[lane] = px;
          // new ports and objectives, committed only if every system's m x m system is regular
          for (int sy = 0; sy < g.n_sys && !bad; ++sy) {
            c128 o[kMaxPorts];
            FOR_PORTS(p, g.sys[sy].n_o) o[p] = s_o[sy][p];
            if (!accept_pivot_sys(g.sys[sy], px, m, s_acc_buf, s_z[sy], s_y[sy], s_tz[sy], o)) bad = 1;
            if (lane == 0) {
              FOR_PORTS(p, g.sys[sy].n_o) s_o_new[sy][p] = o[p];
              s_f_new[sy] = objective_of(g.sys[sy].op, o);
            }
          }
          if (lane == 0 && !bad) {
            for (int sy = 0; sy < g.n_sys; ++sy) {
              FOR_PORTS(p, g.sys[sy].n_o) s_o[sy][p] = s_o_new[sy][p];
              s_f[sy] = s_f_new[sy];
            }
            s_m = m;
            s_F = combine_of(s_f, g.n_sys, g.combine, g.kind);
          }
        }
      }
      if (lane == 0) {
        s_k = k;
        s_pos = pos_k;
        s_bad = bad;
      }
    }
    __syncthreads();
    slot ^= 1;
    ++rd;
    const int k = s_k, pos_k = s_pos;
    if (k == -2 || s_bad) {  // invalid order entry or tile; a forced tile that is singular
      status = k == -2 ? PNGF_EINVAL : (forced ? PNGF_ESINGULAR : PNGF_EINVAL);
      break;
    }
    if (k < 0) {
      if (g.mode == PNGF_FIRST_IMPROVEMENT) {
        n_evals += nt - t;
        ++sweeps_done;
        if (acc_in_sweep == 0) { converged = 1; break; }
        ++s;
        if (s >= g.n_sweeps) break;
        t = 0;
        acc_in_sweep = 0;
        if (g.order) {
          setup_sweep(s);
          if (!grid_sync(ctl)) { failed = true; break; }
          if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) { status = PNGF_EINVAL; break; }
        }
        continue;
      } else {
        n_evals += nt;
        ++sweeps_done;
        converged = 1;
        break;
      }
    }
    // ---- keep tile k
    if (!isfinite(s_F)) status = PNGF_ENUMERIC;
    if (!forced) {
      if (g.mode == PNGF_FIRST_IMPROVEMENT) {
        n_evals += pos_k - t + 1;
        t = pos_k + 1;
      } else {
        n_evals += nt;
        ++sweeps_done;
      }
    }
    ++acc_in_sweep;
    if (cta == 0 && tid == 0) {
      if (n_acc < g.trace_cap) {
        if (g.trace) {
          int32_t* tr = g.trace + 4 * n_acc;
          tr[0] = g.mode == PNGF_FIRST_IMPROVEMENT ? s : (int)n_acc;
          tr[1] = pos_k;
          tr[2] = k;
          tr[3] = 0;
        }
        if (g.trace_f) g.trace_f[n_acc] = s_F;
      } else if (status == PNGF_OK) {
        status = PNGF_ECAPACITY;
      }
    }
    ++n_acc;
    const int m = s_m;
    // U = W[own, K], V = U Z for every system (W, Z read before any update)
    for (int sy = 0; sy < g.n_sys; ++sy) {
      const SweepArgs& a = g.sys[sy];
      c128* U = g.U + (size_t)sy * n * M;
      c128* V = g.V + (size_t)sy * n * M;
      for (int q = tid; q < (pe - pb) * m; q += blockDim.x) {
        const int j = pb + q / m, c = q % m;
        U[(size_t)j * M + c] = w_sym(a, j, s_px[c]);
      }
      __syncthreads();
      for (int q = tid; q < (pe - pb) * m; q += blockDim.x) {
        const int j = pb + q / m, c = q % m;
        c128 acc = mk(0.0, 0.0);
        for (int b = 0; b < m; ++b) acc = cfma(U[(size_t)j * M + b], s_z[sy][b * kTileMax + c], acc);
        V[(size_t)j * M + c] = acc;
      }
    }
    if (!grid_sync(ctl)) { failed = true; break; }
    // rank-m update of the upper triangle and the state of the own pixels
    for (int sy = 0; sy < g.n_sys; ++sy) {
      const SweepArgs& a = g.sys[sy];
      const c128* U = g.U + (size_t)sy * n * M;
      const c128* V = g.V + (size_t)sy * n * M;
      long long e = eb + tid;
      if (e < ee) {
        int i, j;
        tri_rc(e, n, i, j);
        for (; e < ee; e += blockDim.x) {
          c128* w = a.W + (size_t)i * a.ldw + j;
          c128 acc = *w;
          for (int c = 0; c < m; ++c) acc = cfma(V[(size_t)i * M + c], U[(size_t)j * M + c], acc);
          *w = acc;
          tri_step(i, j, n, blockDim.x);
        }
      }
      for (int j = pb + tid; j < pe; j += blockDim.x) {
        c128 dj = a.diag[j], ej = a.e[j];
        for (int c = 0; c < m; ++c) {
          const c128 u = U[(size_t)j * M + c];
          dj = cfma(V[(size_t)j * M + c], u, dj);
          ej = cfma(u, s_y[sy][c], ej);
        }
        a.diag[j] = dj;
        a.e[j] = ej;
#pragma unroll 1
        for (int p = 0; p < a.n_o; ++p) {
          c128* tp = a.T + (size_t)p * a.ldt + j;
          c128 acc = *tp;
          for (int c = 0; c < m; ++c) acc = cfma(s_tz[sy][p * kTileMax + c], U[(size_t)j * M + c], acc);
          *tp = acc;
        }
      }
      // the tile's pixels flip (b and v), pixel by pixel in the owner's range
      if (tid < m) {
        const int k2 = s_px[tid];
        if (k2 >= pb && k2 < pe) {
          const uint8_t nb = a.b[k2] ^ 1;
          a.b[k2] = nb;
          a.v[k2] = nb ? a.dv[k2] : mk(0.0, 0.0);
        }
      }
    }
    if (!grid_sync(ctl)) { failed = true; break; }
    ++since_refresh;
    if (g.refresh_k > 0 && since_refresh >= g.refresh_k) {
      since_refresh = 0;
      ++n_refresh;
      int* act_smem = reinterpret_cast<int*>(gen_smem);
      for (int sy = 0; sy < g.n_sys && !failed; ++sy) {
        const SweepArgs& a = g.sys[sy];
        refresh_x(a, pb, pe);
        if (!grid_sync(ctl)) { failed = true; break; }
        const int m_act = refresh_residual(a, pb, pe, act_smem);
        sum_active += m_act;
        const int t_end = count_below(act_smem, m_act, pe - 1);
        if (!grid_sync(ctl)) { failed = true; break; }
        correct_strips<false>(a, pb, pe, a.actg, t_end, reinterpret_cast<float*>(act_smem),
                              (int)dynamic_smem_bytes());
        if (!grid_sync(ctl)) { failed = true; break; }
        ports_partial(a, pb, pe);
        if (!grid_sync(ctl)) { failed = true; break; }
        ports_total(a, s_o[sy]);
        if (tid == 0) s_f[sy] = objective_of(a.op, s_o[sy]);
        __syncthreads();
      }
      if (failed) break;
      if (tid == 0) s_F = combine_of(s_f, g.n_sys, g.combine, g.kind);
      __syncthreads();
    }
    if (status == PNGF_ENUMERIC || forced) break;
    if (g.mode == PNGF_BEST_IMPROVEMENT && n_acc >= g.n_sweeps) break;
    if (g.mode == PNGF_FIRST_IMPROVEMENT && t >= nt) {
      ++sweeps_done;
      ++s;
      if (s >= g.n_sweeps) break;
      t = 0;
      acc_in_sweep = 0;
      if (g.order) {
        setup_sweep(s);
        if (!grid_sync(ctl)) { failed = true; break; }
        if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) { status = PNGF_EINVAL; break; }
      }
    }
  }
  if (cta == 0 && tid == 0) {
    if (failed) status = PNGF_ETIMEOUT;
    for (int sy = 0; sy < g.n_sys; ++sy) {
      Control* c = g.sys[sy].ctl;
      FOR_PORTS(p, g.sys[sy].n_o) c->o[p] = s_o[sy][p];
      c->f = s_f[sy];
      c->since_refresh = since_refresh;
      c->n_acc_total += (int)n_acc;
    }
    const long long cnt[8] = {n_acc, n_evals, sweeps_done, converged, n_refresh, 0, status, sum_active};
    for (int q = 0; q < 8; ++q) ctl->counters[q] = cnt[q];
    if (g.counters)
      for (int q = 0; q < 8; ++q) g.counters[q] = cnt[q];
    if (status == PNGF_ENUMERIC || status == PNGF_ETIMEOUT || status == PNGF_EINVAL || status == PNGF_ESINGULAR)
      latch_status(ctl, status);
  }
}

// single call: the combined objective of every listed tile (one warp per tile)
__global__ void __launch_bounds__(256) score_tiles_kernel(const __grid_constant__ GenArgs g, const int* __restrict__ list,
                                                          int count, double* __restrict__ F_out,
                                                          double* __restrict__ f_sys_out) {
  extern __shared__ __align__(16) unsigned char sc_smem[];
  __shared__ c128 s_o[kMaxSys][kMaxPorts];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0)
    for (int s = 0; s < g.n_sys; ++s) FOR_PORTS(p, g.sys[s].n_o) s_o[s][p] = g.sys[s].ctl->o[p];
  __syncthreads();
  c128* wbuf = reinterpret_cast<c128*>(sc_smem) + (size_t)warp * kTileMax * kScoreLd;
  for (int i = blockIdx.x * nw + warp; i < count; i += gridDim.x * nw) {
    const int ti = list[i];
    double F = NAN, fs[kMaxSys];
    bool ok = ti >= 0 && ti < g.n_tiles && score_tile(g, s_o, ti, wbuf, F, fs);
    if (lane == 0) {
      F_out[i] = ok ? F : NAN;
      if (f_sys_out)
        for (int s = 0; s < g.n_sys; ++s) f_sys_out[(size_t)i * g.n_sys + s] = ok ? fs[s] : NAN;
    }
  }
}

size_t tiles_smem(int n) {
  const size_t score = (size_t)kWarps * kTileMax * kScoreLd * sizeof(c128);
  const size_t act = (size_t)n * sizeof(int), ct = (size_t)110 * 1024;
  size_t r = act > ct ? act : ct;
  return r > score ? r : score;
}

}  // namespace

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

size_t tiles_workspace_bytes(int n_sys, int n_d, int n_tiles, int tile_m) {
  const size_t uv = (size_t)n_sys * n_d * tile_m * sizeof(c128);
  return 2 * align256(uv) + align256((size_t)n_tiles * sizeof(int)) + 2 * align256((size_t)2 * 1024 * 8);
}

static pngf_status make_gen(pngf_ctx* const* ctxs, int n_sys, int combine, const int32_t* tiles, int n_tiles,
                            int tile_m, void* ws, GenArgs& g) {
  g = GenArgs{};
  for (int s = 0; s < n_sys; ++s) g.sys[s] = make_args(ctxs[s]);
  g.n_sys = n_sys;
  g.combine = combine;
  g.kind = ctxs[0]->cfg.objective;
  g.tiles = tiles;
  g.n_tiles = n_tiles;
  g.tile_m = tile_m;
  const int n = ctxs[0]->cfg.n_d;
  char* w = static_cast<char*>(ws);
  const size_t uv = align256((size_t)n_sys * n * tile_m * sizeof(c128));
  g.U = reinterpret_cast<c128*>(w);
  g.V = reinterpret_cast<c128*>(w + uv);
  g.pos_of = reinterpret_cast<int*>(w + 2 * uv);
  g.part_gain = reinterpret_cast<double*>(w + 2 * uv + align256((size_t)n_tiles * sizeof(int)));
  g.part_key = reinterpret_cast<long long*>(reinterpret_cast<char*>(g.part_gain) + align256((size_t)2 * 1024 * 8));
  g.mode = ctxs[0]->cfg.mode;
  g.refresh_k = ctxs[0]->cfg.refresh_k;
  g.tau = ctxs[0]->cfg.tau;
  g.forced_tile = -1;
  return PNGF_OK;
}

static int tiles_grid(pngf_ctx* c) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(dbs_tiles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tiles_smem(32768));
    cudaFuncSetAttribute(score_tiles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((256 / 32) * kTileMax * kScoreLd * sizeof(c128)));
    attr = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dbs_tiles_kernel, kThreads, tiles_smem(c->cfg.n_d));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;
  int g = c->n_sm * per_sm;
  if (c->cfg.n_ctas > 0 && c->cfg.n_ctas < g) g = c->cfg.n_ctas;
  if (g > 1024) g = 1024;
  return g;
}

pngf_status run_sweep_tiles(pngf_ctx* const* ctxs, int n_sys, int combine, const int32_t* tiles, int n_tiles,
                            int tile_m, int n_sweeps, const int32_t* order, int forced_tile, int32_t* trace,
                            double* trace_f, int32_t trace_cap, int64_t* counters, void* ws) {
  pngf_ctx* c0 = ctxs[0];
  GenArgs g;
  make_gen(ctxs, n_sys, combine, tiles, n_tiles, tile_m, ws, g);
  g.n_sweeps = n_sweeps;
  g.order = order;
  g.forced_tile = forced_tile;
  g.trace = trace;
  g.trace_f = trace_f;
  g.trace_cap = trace_cap;
  g.counters = counters;
  Control* ctl = g.sys[0].ctl;
  if (cudaMemsetAsync(&ctl->bar_count, 0, 2 * sizeof(unsigned), c0->stream) != cudaSuccess ||
      cudaMemsetAsync(&ctl->sel[0], 0xff, sizeof(ctl->sel), c0->stream) != cudaSuccess)
    return PNGF_ECUDA;
  const int grid = tiles_grid(c0);
  void* params[] = {&g};
  return cuda_status(cudaLaunchCooperativeKernel((const void*)dbs_tiles_kernel, dim3(grid), dim3(kThreads), params,
                                                 tiles_smem(c0->cfg.n_d), c0->stream));
}

pngf_status score_tiles(pngf_ctx* const* ctxs, int n_sys, int combine, const int32_t* tiles, int n_tiles,
                        int tile_m, const int32_t* list, int count, double* F, double* f_sys, void* ws) {
  if (count <= 0) return PNGF_OK;
  pngf_ctx* c0 = ctxs[0];
  GenArgs g;
  make_gen(ctxs, n_sys, combine, tiles, n_tiles, tile_m, ws, g);
  tiles_grid(c0);
  int blocks = (count + 7) / 8;
  if (blocks > 4 * c0->n_sm) blocks = 4 * c0->n_sm;
  score_tiles_kernel<<<blocks, 256, (256 / 32) * kTileMax * kScoreLd * sizeof(c128), c0->stream>>>(g, list, count,
                                                                                                  F, f_sys);
  return cuda_status(cudaGetLastError());
}

}  // namespace pngf
