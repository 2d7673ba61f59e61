// Direct binary search over perfect-conductor (PEC) pixels: the paper's own
// binary system, Eq. 2, [(I - P) + P G] j = P e_inc, in this code's sign of G
// (total field e = c_d + G j; on a metal pixel e = 0, on an empty one j = 0).
//
// For metal set M the solution is j_M = -(G_MM)^-1 c_M.  The search keeps
//   H = (G_MM)^-1 padded with zeros (complex symmetric),
//   Q = G H,  W = G - G H G (complex symmetric, zero on M: the field-form
//   inverse of the lossy system in the limit of infinite contrast),
//   e = c_d + G j (total field), j, T = G_od - G_od H G, R = G_od H,
//   diag W, diag H, o = c_o + G_od j.
// A flip is a rank-1 change of the metal set (the rank-1 case of the
// paper's Woodbury update, Eq. 9, for dP = +-e_k e_k^T, scored by Eq. 14):
//   add k (empty -> metal): x = W[:, k], y = e_k - Q[k, :]^T, s = W_kk,
//     W -= x x^T/s, H += y y^T/s, Q += x y^T/s, gamma = e_k / s, P_k = T[:, k]
//   remove k (metal -> empty): x = Q[:, k], y = H[:, k], s = H_kk,
//     W += x x^T/s, H -= y y^T/s, Q -= x y^T/s, gamma = j_k / s, P_k = R[:, k]
// and in both cases e -= gamma x, j -= gamma y, o -= gamma P_k,
// T += aW P_k x^T, R += aH P_k y^T, diag W += aW x.x, diag H += aH y.y with
// (aW, aH) = (-1/s, 1/s) for an add and (1/s, -1/s) for a removal.  A
// candidate is scored from o - gamma_k P_k alone (O(n_o)).
//
// The initial state of a design is built from the empty design (W = G,
// everything else zero or the incident field) by adding its metal pixels one
// by one with the same update (pngf_factor); the search is one cooperative
// launch with the FP64 path's selection and barriers.
#include <cstdio>

#include "sweep_common.cuh"

namespace pngf {
namespace {

struct PecArgs {
  SweepArgs a;  // W, diag (= diag W), e (total field), T, b, cbuf (x), ctl, ...
  c128* H;
  c128* Q;  // n x ldw, full
  c128* j;
  c128* R;  // n_o x ldt
  c128* diagH;
  c128* ybuf;  // n
  const int* forced;  // forced list of pixels to flip in order (factor), or nullptr
  int n_forced;
};

struct PecPivot {
  int k, add;
  c128 s_inv, gamma;  // 1/s, gamma = (add ? e_k : j_k) / s
  c128 Pk[kMaxPorts];  // T[:, k] (add) or R[:, k] (remove)
};

__device__ __forceinline__ c128 sym_at(const c128* M, int ld, int i, int j) {
  return i <= j ? M[(size_t)i * ld + j] : M[(size_t)j * ld + i];
}

// candidate objective of flipping pixel i; false if its pivot is below 1e-14
__device__ __forceinline__ bool pec_score(const PecArgs& g, const ObjParams& op, int i, const c128* o, double& f) {
  const SweepArgs& a = g.a;
  const bool add = a.b[i] == 0;
  const c128 s = add ? a.diag[i] : g.diagH[i];
  if (cabs2(s) < 1e-28) return false;
  const c128 gam = cdiv(add ? a.e[i] : g.j[i], s);
  const c128* P = add ? a.T : g.R;
  double fn = 0.0;
#pragma unroll 1
  for (int p = 0; p < a.n_o; ++p) fn += objective_term(op, p, cfms(gam, P[(size_t)p * a.ldt + i], o[p]));
  f = fn;
  return true;
}

__device__ __forceinline__ bool pec_pivot(const PecArgs& g, int k, PecPivot& pv) {
  const SweepArgs& a = g.a;
  pv.k = k;
  pv.add = a.b[k] == 0;
  const c128 s = pv.add ? a.diag[k] : g.diagH[k];
  if (cabs2(s) < 1e-28) return false;
  pv.s_inv = cdiv(mk(1.0, 0.0), s);
  pv.gamma = cmul(pv.add ? a.e[k] : g.j[k], pv.s_inv);
  const c128* P = pv.add ? a.T : g.R;
  FOR_PORTS(p, a.n_o) pv.Pk[p] = P[(size_t)p * a.ldt + k];
  return true;
}

// x (cbuf) and y (ybuf) of the kept flip for pixels [pb, pe)
__device__ void pec_gather(const PecArgs& g, const PecPivot& pv, int pb, int pe) {
  const SweepArgs& a = g.a;
  const int k = pv.k;
  for (int i = pb + threadIdx.x; i < pe; i += blockDim.x) {
    if (pv.add) {
      a.cbuf[i] = sym_at(a.W, a.ldw, i, k);
      const c128 q = g.Q[(size_t)k * a.ldw + i];
      g.ybuf[i] = i == k ? mk(1.0 - q.x, -q.y) : mk(-q.x, -q.y);
    } else {
      a.cbuf[i] = g.Q[(size_t)i * a.ldw + k];
      g.ybuf[i] = sym_at(g.H, a.ldw, i, k);
    }
  }
}

// the rank-1 updates of W and H on elements [eb, ee) of their upper
// triangles, of the rows [pb, pe) of Q, and the state of pixels [pb, pe)
__device__ void pec_update(const PecArgs& g, const PecPivot& pv, int pb, int pe, long long eb, long long ee) {
  const SweepArgs& a = g.a;
  const int n = a.n;
  const c128 aW = pv.add ? mk(-pv.s_inv.x, -pv.s_inv.y) : pv.s_inv;
  const c128 aH = mk(-aW.x, -aW.y);
  const c128* x = a.cbuf;
  const c128* y = g.ybuf;
  long long e = eb + threadIdx.x;
  if (e < ee) {
    int i, j;
    tri_rc(e, n, i, j);
    for (; e < ee; e += blockDim.x) {
      const size_t o = (size_t)i * a.ldw + j;
      a.W[o] = cfma(cmul(aW, x[i]), x[j], a.W[o]);
      g.H[o] = cfma(cmul(aH, y[i]), y[j], g.H[o]);
      tri_step(i, j, n, blockDim.x);
    }
  }
  for (int i = pb; i < pe; ++i) {
    const c128 xi = cmul(aH, x[i]);  // aQ = aH (= +1/s for an add, -1/s for a removal)
    c128* qrow = g.Q + (size_t)i * a.ldw;
    for (int c = threadIdx.x; c < n; c += blockDim.x) qrow[c] = cfma(xi, y[c], qrow[c]);
  }
  for (int i = pb + threadIdx.x; i < pe; i += blockDim.x) {
    const c128 xi = x[i], yi = y[i];
    a.e[i] = cfms(pv.gamma, xi, a.e[i]);
    g.j[i] = cfms(pv.gamma, yi, g.j[i]);
    a.diag[i] = cfma(cmul(aW, xi), xi, a.diag[i]);
    g.diagH[i] = cfma(cmul(aH, yi), yi, g.diagH[i]);
    const c128 wx = cmul(aW, xi), hy = cmul(aH, yi);
#pragma unroll 1
    for (int p = 0; p < a.n_o; ++p) {
      c128* t = a.T + (size_t)p * a.ldt + i;
      c128* r = g.R + (size_t)p * a.ldt + i;
      *t = cfma(wx, pv.Pk[p], *t);
      *r = cfma(hy, pv.Pk[p], *r);
    }
    if (i == pv.k) a.b[i] ^= 1;
  }
}

__global__ void __launch_bounds__(kThreads) dbs_pec_kernel(const __grid_constant__ PecArgs g) {
  const SweepArgs& a = g.a;
  const int P = gridDim.x, cta = blockIdx.x;
  const int n = a.n;
  const int pb = (int)((long long)n * cta / P), pe = (int)((long long)n * (cta + 1) / P);
  const long long E = (long long)n * (n + 1) / 2;
  const long long eb = E * cta / P, ee = E * (cta + 1) / P;
  Control* ctl = a.ctl;
  hold_if_asked(ctl);
  __shared__ c128 s_o[kMaxPorts];
  __shared__ double s_f;
  __shared__ PecPivot s_pv;
  __shared__ int s_k, s_pos, s_bad;
  __shared__ ObjParams s_op;
  if (threadIdx.x == 0) {
    s_op = a.op;
    FOR_PORTS(p, a.n_o) s_o[p] = ctl->o[p];
    s_f = ctl->f;
  }
  __syncthreads();
  long long n_acc = 0, n_evals = 0;
  int sweeps_done = 0, converged = 0, status = PNGF_OK;
  int s = 0, t = 0, acc_in_sweep = 0, slot = 0, rd = 0;
  bool failed = false;
  const bool forced = g.forced != nullptr;
  auto setup_sweep = [&](int sw) {
    if (a.order)
      for (int q = pb + threadIdx.x; q < pe; q += blockDim.x) {
        const int px = a.order[(size_t)sw * n + q];
        if ((unsigned)px < (unsigned)n) a.pos_of[px] = q;
        else latch_status(ctl, PNGF_EINVAL);
      }
  };
  if (!forced && a.mode == PNGF_FIRST_IMPROVEMENT && a.order) {
    setup_sweep(0);
    if (!grid_sync(ctl)) failed = true;
    else if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) status = PNGF_EINVAL;
  }
  int fi = 0;  // next entry of the forced list
  // PNGF_ECAPACITY (set by CTA 0 alone) must not end one CTA's loop before the others'
  while (!failed && (status == PNGF_OK || status == PNGF_ECAPACITY)) {
    const double f = s_f;
    const double thr = accept_threshold(s_op, f);
    if (forced) {
      if (fi >= g.n_forced) break;
    } else if (a.mode == PNGF_FIRST_IMPROVEMENT) {
      long long best = LLONG_MAX;
      for (int i = pb + threadIdx.x; i < pe; i += blockDim.x) {
        const int pos = a.order ? a.pos_of[i] : i;
        if (pos < t) continue;
        double fn;
        if (!pec_score(g, s_op, i, s_o, fn)) continue;
        if (gain_of(s_op, fn, f) - thr > 0.0 && pos < best) best = pos;
      }
      best = block_min_ll(best);
      if (threadIdx.x == 0) sel_offer(ctl, rd, best, cta);
      if (!grid_sync(ctl)) { failed = true; break; }
    } else {
      double gb = -INFINITY;
      int pix = INT_MAX;
      for (int i = pb + threadIdx.x; i < pe; i += blockDim.x) {
        double fn;
        if (!pec_score(g, s_op, i, s_o, fn)) continue;
        const double gg = gain_of(s_op, fn, f);
        if (better(gg, i, gb, pix)) { gb = gg; pix = i; }
      }
      block_best(gb, pix);
      if (threadIdx.x == 0) {
        a.part_gain[slot * P + cta] = gb;
        a.part_key[slot * P + cta] = pix;
      }
      if (!grid_sync(ctl)) { failed = true; break; }
    }
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      int k = -1, pos_k = -1;
      if (forced) {
        k = g.forced[fi];
        if ((unsigned)k >= (unsigned)n) k = -2;
        pos_k = fi;
      } else if (a.mode == PNGF_FIRST_IMPROVEMENT) {
        const unsigned long long key = sel_read(ctl, rd);
        if (key != ~0ull) {
          pos_k = (int)(key >> 10);
          k = a.order ? a.order[(size_t)s * n + pos_k] : pos_k;
          if ((unsigned)k >= (unsigned)n) k = -2;
        }
      } else {
        double gb = -INFINITY;
        int pix = INT_MAX;
        for (int q = lane; q < P; q += 32) {
          const double gg = a.part_gain[slot * P + q];
          const int pp = (int)a.part_key[slot * P + q];
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
      if (lane == 0) {
        int bad = 0;
        if (k >= 0) {
          if (!pec_pivot(g, k, s_pv)) {
            bad = 1;
          } else {
            FOR_PORTS(p, a.n_o) s_o[p] = cfms(s_pv.gamma, s_pv.Pk[p], s_o[p]);
            s_f = objective_of(s_op, s_o);
          }
        }
        s_k = k;
        s_pos = pos_k;
        s_bad = bad;
      }
    }
    __syncthreads();
    slot ^= 1;
    ++rd;
    const int k = s_k, pos_k = s_pos;
    if (k == -2) { status = PNGF_EINVAL; break; }
    if (s_bad) { status = PNGF_ESINGULAR; break; }  // only a forced flip can meet a zero pivot
    if (k < 0) {
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
          if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) { status = PNGF_EINVAL; break; }
        }
        continue;
      } else {
        n_evals += n;
        ++sweeps_done;
        converged = 1;
        break;
      }
    }
    if (!isfinite(s_f)) status = PNGF_ENUMERIC;
    if (forced) {
      ++fi;
    } else {
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
    }
    pec_gather(g, s_pv, pb, pe);
    if (!grid_sync(ctl)) { failed = true; break; }
    pec_update(g, s_pv, pb, pe, eb, ee);
    if (!grid_sync(ctl)) { failed = true; break; }
    if (status == PNGF_ENUMERIC) break;
    if (!forced && a.mode == PNGF_BEST_IMPROVEMENT && n_acc >= a.n_sweeps) break;
    if (!forced && a.mode == PNGF_FIRST_IMPROVEMENT && t >= n) {
      ++sweeps_done;
      ++s;
      if (s >= a.n_sweeps) break;
      t = 0;
      acc_in_sweep = 0;
      if (a.order) {
        setup_sweep(s);
        if (!grid_sync(ctl)) { failed = true; break; }
        if (*reinterpret_cast<volatile int*>(&ctl->status) == PNGF_EINVAL) { status = PNGF_EINVAL; break; }
      }
    }
  }
  if (cta == 0 && threadIdx.x == 0) {
    if (failed) status = PNGF_ETIMEOUT;
    FOR_PORTS(p, a.n_o) ctl->o[p] = s_o[p];
    ctl->f = s_f;
    if (!forced) {
      ctl->n_acc_total += (int)n_acc;
      const long long cnt[8] = {n_acc, n_evals, sweeps_done, converged, 0, 0, status, 0};
      for (int q = 0; q < 8; ++q) ctl->counters[q] = cnt[q];
      if (a.counters)
        for (int q = 0; q < 8; ++q) a.counters[q] = cnt[q];
    }
    if (status != PNGF_OK && status != PNGF_ECAPACITY) latch_status(ctl, status);
  }
}

// the empty design's state: W = G (upper triangle), H = Q = 0, e = c_d,
// j = 0, T = G_od, R = 0, diag W = diag G, diag H = 0, b = 0
__global__ void pec_empty_kernel(const __grid_constant__ PecArgs g) {
  const SweepArgs& a = g.a;
  const int n = a.n;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const size_t o = (size_t)i * a.ldw + c;
      a.W[o] = c >= i ? a.G[(size_t)i * n + c] : mk(0.0, 0.0);
      g.H[o] = mk(0.0, 0.0);
      g.Q[o] = mk(0.0, 0.0);
    }
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    a.diag[i] = a.G[(size_t)i * n + i];
    a.e[i] = a.cd[i];
    g.j[i] = mk(0.0, 0.0);
    g.diagH[i] = mk(0.0, 0.0);
    a.b[i] = 0;
    a.v[i] = mk(0.0, 0.0);
    for (int p = 0; p < a.n_o; ++p) {
      a.T[(size_t)p * a.ldt + i] = a.God[(size_t)p * n + i];
      g.R[(size_t)p * a.ldt + i] = mk(0.0, 0.0);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Control* ctl = a.ctl;
    FOR_PORTS(p, a.n_o) ctl->o[p] = a.co[p];
    ctl->f = objective_of(a.op, a.co);
    ctl->since_refresh = 0;
    ctl->n_acc_total = 0;
  }
}

// forced list of the metal pixels of design b (ascending), and its length
__global__ void pec_list_kernel(const uint8_t* __restrict__ b, int n, int* list, int* count) {
  __shared__ int s_base;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  for (int i0 = 0; i0 < n; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const int on = i < n && b[i] != 0;
    // block-wide exclusive scan of `on` in thread order (one block)
    __shared__ int s_cnt[1024];
    s_cnt[threadIdx.x] = on;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      const int v = threadIdx.x >= (unsigned)off ? s_cnt[threadIdx.x - off] : 0;
      __syncthreads();
      s_cnt[threadIdx.x] += v;
      __syncthreads();
    }
    if (on) list[s_base + s_cnt[threadIdx.x] - 1] = i;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_base += s_cnt[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = s_base;
}

__global__ void pec_score_kernel(const __grid_constant__ PecArgs g, const int32_t* __restrict__ pixels, int m,
                                  double* __restrict__ f_new) {
  __shared__ ObjParams s_op;
  __shared__ c128 o[kMaxPorts];
  if (threadIdx.x == 0) {
    s_op = g.a.op;
    FOR_PORTS(p, g.a.n_o) o[p] = g.a.ctl->o[p];
  }
  __syncthreads();
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
    const int i = pixels[q];
    double fn = NAN;
    const bool ok = i >= 0 && i < g.a.n && pec_score(g, s_op, i, o, fn);
    f_new[q] = ok ? fn : NAN;
  }
}

}  // namespace

static PecArgs make_pec(pngf_ctx* c) {
  PecArgs g{};
  g.a = make_args(c);
  const Layout& L = c->L;
  g.H = at<c128>(c, L.LU);
  g.Q = at<c128>(c, L.Q);
  g.j = at<c128>(c, L.pj);
  g.R = at<c128>(c, L.pR);
  g.diagH = at<c128>(c, L.pdiagH);
  g.ybuf = at<c128>(c, L.rbuf);
  return g;
}

static int pec_grid(pngf_ctx* c) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dbs_pec_kernel, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;
  int g = c->n_sm * per_sm;
  if (c->cfg.n_ctas > 0 && c->cfg.n_ctas < g) g = c->cfg.n_ctas;
  if (g > c->L.n_part) g = c->L.n_part;
  return g;
}

static pngf_status launch_pec(pngf_ctx* c, PecArgs& g) {
  Control* ctl = g.a.ctl;
  if (cudaMemsetAsync(&ctl->bar_count, 0, 2 * sizeof(unsigned), c->stream) != cudaSuccess ||
      cudaMemsetAsync(&ctl->sel[0], 0xff, sizeof(ctl->sel), c->stream) != cudaSuccess)
    return PNGF_ECUDA;
  void* params[] = {&g};
  return cuda_status(cudaLaunchCooperativeKernel((const void*)dbs_pec_kernel, dim3(pec_grid(c)), dim3(kThreads),
                                                 params, 0, c->stream));
}

pngf_status factor_pec(pngf_ctx* c, const uint8_t* b) {
  PecArgs g = make_pec(c);
  const int n = c->cfg.n_d;
  int blocks = n < 4 * c->n_sm ? n : 4 * c->n_sm;
  pec_empty_kernel<<<blocks, 256, 0, c->stream>>>(g);
  int* list = at<int>(c, c->L.pos_of);  // scratch until the search sets it
  int* count = at<int>(c, c->L.actg);
  pec_list_kernel<<<1, 1024, 0, c->stream>>>(b, n, list, count);
  if (cudaGetLastError() != cudaSuccess) return PNGF_ECUDA;
  int h_count = 0;
  if (cudaMemcpyAsync(&h_count, count, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return PNGF_ECUDA;
  if (h_count == 0) return PNGF_OK;
  g.forced = list;
  g.n_forced = h_count;
  return launch_pec(c, g);
}

pngf_status run_sweep_pec(pngf_ctx* c, int n_sweeps, const int32_t* order, int32_t* trace, double* trace_f,
                          int32_t trace_cap, int64_t* counters) {
  PecArgs g = make_pec(c);
  g.a.n_sweeps = n_sweeps;
  g.a.order = order;
  g.a.trace = trace;
  g.a.trace_f = trace_f;
  g.a.trace_cap = trace_cap;
  g.a.counters = counters;
  return launch_pec(c, g);
}

pngf_status accept_flip_pec(pngf_ctx* c, int pixel) {
  PecArgs g = make_pec(c);
  int* one = at<int>(c, c->L.actg);  // scratch: a one-entry forced list
  if (cudaMemcpyAsync(one, &pixel, sizeof(int), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return PNGF_ECUDA;
  g.forced = one;
  g.n_forced = 1;
  pngf_status st = launch_pec(c, g);
  if (st != PNGF_OK) return st;
  // the pageable source of the copy above must outlive it
  return cuda_status(cudaStreamSynchronize(c->stream));
}

pngf_status score_flips_pec(pngf_ctx* c, const int32_t* pixels, int m, double* f_new) {
  if (m <= 0) return PNGF_OK;
  PecArgs g = make_pec(c);
  int blocks = (m + 255) / 256;
  if (blocks > 4 * c->n_sm) blocks = 4 * c->n_sm;
  pec_score_kernel<<<blocks, 256, 0, c->stream>>>(g, pixels, m, f_new);
  return cuda_status(cudaGetLastError());
}

}  // namespace pngf
