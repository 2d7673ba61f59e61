// Internal declarations shared by the PNGF CUDA translation units.
//
// Layout of the caller's workspace (all offsets 256-byte aligned), for one
// design region of n = n_d pixels and n_o ports:
//   W        c128 n x ldw        maintained inverse W = M^-1 G (FP64 path; the
//                                 upper triangle j >= i is kept current, W is
//                                 complex symmetric).  Also the LU factors'
//                                 right-hand side during pngf_factor.
//   LU       c128 n x ldw        LU factors of M (factor only)
//   Wlo_re,
//   Wlo_im   f32  n x ldl each   planar FP32 copy of W for the mixed path
//   X        c128 n x R          delayed columns c_i of the mixed path
//   xa       c128 R              their coefficients alpha_i
//   state    diag(W), e, T (n_o x ldt), v, b, pos_of, scratch vectors
//   snap     copy of W (or Wlo) and state for pngf_snapshot / pngf_restore
//   ctl      control block (status latch, counters)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pngf.h"

namespace pngf {

// ---------------------------------------------------------------- complex
struct __align__(16) c128 {
  double x, y;
};

__host__ __device__ __forceinline__ c128 mk(double a, double b) { return c128{a, b}; }
__host__ __device__ __forceinline__ c128 cadd(c128 a, c128 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ c128 csub(c128 a, c128 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ c128 cmul(c128 a, c128 b) {
  return mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a*b + c with four fused multiply-adds
__host__ __device__ __forceinline__ c128 cfma(c128 a, c128 b, c128 c) {
  return mk(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// c - a*b
__host__ __device__ __forceinline__ c128 cfms(c128 a, c128 b, c128 c) {
  return mk(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ double cabs2(c128 a) { return fma(a.x, a.x, a.y * a.y); }
__host__ __device__ __forceinline__ double cabs1(c128 a) { return fabs(a.x) + fabs(a.y); }
// a / b by Smith's scaling (no overflow for |b| spanning the double range)
__host__ __device__ __forceinline__ c128 cdiv(c128 a, c128 b) {
  if (fabs(b.y) <= fabs(b.x)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return mk((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  }
  double r = b.x / b.y, den = b.y + b.x * r;
  return mk((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}

// ---------------------------------------------------------------- objective
constexpr int kMaxPorts = PNGF_MAX_PORTS;
// Loop over the ports with a compile-time trip count so that per-port arrays
// stay in registers.
#define FOR_PORTS(p, n) _Pragma("unroll") for (int p = 0; p < kMaxPorts; ++p) if (p < (n))

struct ObjParams {
  int n_o;
  int kind;  // pngf_objective
  double tau;
  double w[kMaxPorts];
  c128 off[kMaxPorts];
  c128 scale[kMaxPorts];
};

// Contribution of port p to the objective (Supplementary Note 9 style):
// w_p |S_p|^2 (maximised) or w_p (1 - |S_p|)^2 (minimised), S_p = (o_p - off_p) scale_p.
__device__ __forceinline__ double objective_term(const ObjParams& op, int p, c128 o) {
  c128 s = cmul(csub(o, op.off[p]), op.scale[p]);
  double a2 = cabs2(s);
  if (op.kind == PNGF_OBJ_MAX_WEIGHTED_POWER) return op.w[p] * a2;
  double m = 1.0 - sqrt(a2);
  return op.w[p] * (m * m);
}

__device__ __forceinline__ double objective_of(const ObjParams& op, const c128* o) {
  double f = 0.0;
  FOR_PORTS(p, op.n_o) f += objective_term(op, p, o[p]);
  return f;
}
// signed improvement, positive = better
__device__ __forceinline__ double gain_of(const ObjParams& op, double f_new, double f_old) {
  return op.kind == PNGF_OBJ_MAX_WEIGHTED_POWER ? f_new - f_old : f_old - f_new;
}
__device__ __forceinline__ double accept_threshold(const ObjParams& op, double f) {
  return op.tau * fmax(fabs(f), 1e-30);
}

// bytes per candidate-record slot ([2][grid] slots in the workspace)
constexpr int kRecordBytes = 512;

// ---------------------------------------------------------------- control block
// Device-resident, inside the workspace.
struct Control {
  int status;            // latched pngf_status (first error wins)
  int hold_cta;          // failure-detection test hook: CTA hold_cta - 1 of the next sweep waits
                         // (bounded) for hold_flag before it joins the others; 0 = none
  unsigned int bar_count;   // grid barrier arrivals
  unsigned int bar_gen;     // grid barrier generation
  long long counters[8];    // see pngf_dbs_sweep
  unsigned long long sel[3];  // FIRST mode: per-round minimum of (position << 10 | cta), 3 rotating cells
  long long phase_cycles[16];  // SM cycles of CTA 0 per sweep phase (last sweep)
  unsigned long long spin_limit;  // polls before a bounded device wait gives up (0 = default)
  int hold_flag;            // never set: the held CTA's wait runs out
  int pad1;
  double f;                 // current objective
  int factored;
  int n_acc_total;          // accepted flips since the last factor / restore
  int since_refresh;        // accepts since the last refresh
  int r_delay;              // mixed path: columns held in X
  c128 o[kMaxPorts];        // current port amplitudes
};

__device__ __forceinline__ void latch_status(Control* ctl, int s) {
  atomicCAS(&ctl->status, 0, s);
}

// ---------------------------------------------------------------- context
struct Layout {
  size_t W, LU, Q, pj, pR, pdiagH, Wlo_re, Wlo_im, X, xa, diag, e, T, v, b, pos_of, scr, part, rec, slots, actg, gsum, gsplit, xs, xadd, cbuf, ipiv, rbuf,
      snapW, snapState, ctl, total;
  size_t snapW_bytes;  // bytes of the maintained inverse copied by snapshot
  size_t tcimg, tcimgA_bytes, tcimg_bytes;  // mixed path: operand images of the tensor-core fold
  int ldw, ldl, ldt, R, n_part;
  size_t state_bytes;  // contiguous state block [diag .. b] copied by snapshot
};

Layout make_layout(const pngf_config& cfg);

}  // namespace pngf

struct pngf_ctx {
  pngf_config cfg;
  pngf::Layout L;
  cudaStream_t stream;
  const pngf::c128* G;
  const pngf::c128* God;
  const pngf::c128* cd;
  const pngf::c128* co;
  const pngf::c128* dv;
  char* ws;
  pngf::ObjParams obj;
  int n_sm;
  int coop_ctas;  // persistent grid size
  bool factored;
  bool has_snapshot;
  int device;
};

namespace pngf {

template <typename T>
__host__ __forceinline__ T* at(pngf_ctx* c, size_t off) {
  return reinterpret_cast<T*>(c->ws + off);
}

// factor.cu
pngf_status factor_fp64(pngf_ctx* c, const uint8_t* b);
// sweep_mixed.cu
pngf_status mixed_after_factor(pngf_ctx* c);
pngf_status run_sweep_mixed(pngf_ctx* c, int n_sweeps, const int32_t* order, int32_t* trace,
                            double* trace_f, int32_t trace_cap, int64_t* counters);
pngf_status accept_flip_mixed(pngf_ctx* c, int pixel);
// flush_tc.cu
pngf_status flush_tc_launch(pngf_ctx* c);
// batch.cu
size_t batch_workspace_bytes(int n_runs);
pngf_status run_sweep_batch(pngf_ctx* const* ctxs, int n_runs, int n_sweeps, const int32_t* const* orders,
                            int32_t* const* traces, double* const* trace_f, int32_t trace_cap, int64_t* counters,
                            void* ws, size_t ws_bytes);
// sweep.cu
pngf_status run_sweep(pngf_ctx* c, int n_sweeps, const int32_t* order, int32_t* trace,
                      double* trace_f, int32_t trace_cap, int64_t* counters);
pngf_status score_flips(pngf_ctx* c, const int32_t* pixels, int n, double* f_new, double* o_new);
pngf_status accept_flip(pngf_ctx* c, int pixel);
pngf_status accept_flip_noalloc(pngf_ctx* c, int pixel);
pngf_status set_wait_limit(pngf_ctx* c, unsigned long long polls, int hold_plus1);
pngf_status import_finish(pngf_ctx* c, int since_refresh);
// pec.cu
pngf_status factor_pec(pngf_ctx* c, const uint8_t* b);
pngf_status run_sweep_pec(pngf_ctx* c, int n_sweeps, const int32_t* order, int32_t* trace, double* trace_f,
                          int32_t trace_cap, int64_t* counters);
pngf_status accept_flip_pec(pngf_ctx* c, int pixel);
pngf_status score_flips_pec(pngf_ctx* c, const int32_t* pixels, int m, double* f_new);
// gradient.cu
pngf_status gradient(pngf_ctx* c, double* grad, double* dodrho);
// general.cu
size_t tiles_workspace_bytes(int n_sys, int n_d, int n_tiles, int tile_m);
pngf_status run_sweep_tiles(pngf_ctx* const* ctxs, int n_sys, int combine, const int32_t* tiles, int n_tiles,
                            int tile_m, int n_sweeps, const int32_t* order, int forced_tile, int32_t* trace,
                            double* trace_f, int32_t trace_cap, int64_t* counters, void* ws);
pngf_status score_tiles(pngf_ctx* const* ctxs, int n_sys, int combine, const int32_t* tiles, int n_tiles,
                        int tile_m, const int32_t* list, int count, double* F, double* f_sys, void* ws);
int sweep_grid_size(pngf_ctx* c);

inline pngf_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PNGF_OK : PNGF_ECUDA; }

}  // namespace pngf
