// Gradient of the objective with respect to a continuous density of every
// pixel at the current design (Supplementary Note 5, in the field form).
//
// With v_m = rho_m dv_m the chain rule of the note (Wirtinger derivatives of
// a real objective) gives
//   df/drho_m = 2 Re[ sum_p (dphi_p/dS_p) scale_p T[p, m] e_m dv_m ],
// because do/dv_m = T[:, m] e_m (the m-th column of R times the m-th entry
// of the maintained field, the note's elementwise form).  T and e are the
// maintained state, so the gradient costs O(n_o N_d) and reads
// (n_o + 2) x 16 bytes per pixel: one coalesced pass, bound by memory.
#include "sweep_common.cuh"

namespace pngf {
namespace {

__global__ void __launch_bounds__(256) gradient_kernel(SweepArgs a, double* __restrict__ grad,
                                                       c128* __restrict__ dodrho) {
  __shared__ c128 s_c[kMaxPorts];  // (dphi_p/dS_p) scale_p
  if (threadIdx.x == 0) {
    FOR_PORTS(p, a.n_o) {
      const c128 S = cmul(csub(a.ctl->o[p], a.op.off[p]), a.op.scale[p]);
      c128 d;
      if (a.op.kind == PNGF_OBJ_MAX_WEIGHTED_POWER) {
        d = mk(a.op.w[p] * S.x, -a.op.w[p] * S.y);
      } else {
        const double m = sqrt(cabs2(S));
        const double q = m > 0.0 ? -a.op.w[p] * (1.0 - m) / m : 0.0;
        d = mk(q * S.x, -q * S.y);
      }
      s_c[p] = cmul(d, a.op.scale[p]);
    }
  }
  __syncthreads();
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < a.n; m += gridDim.x * blockDim.x) {
    const c128 q = cmul(a.e[m], a.dv[m]);
    double acc = 0.0;
#pragma unroll 1
    for (int p = 0; p < a.n_o; ++p) {
      const c128 d = cmul(a.T[(size_t)p * a.ldt + m], q);
      if (dodrho) dodrho[(size_t)p * a.n + m] = d;
      acc = fma(s_c[p].x, d.x, fma(-s_c[p].y, d.y, acc));
    }
    grad[m] = 2.0 * acc;
  }
}

}  // namespace

pngf_status gradient(pngf_ctx* c, double* grad, double* dodrho) {
  SweepArgs a = make_args(c);
  int blocks = (c->cfg.n_d + 255) / 256;
  if (blocks > 4 * c->n_sm) blocks = 4 * c->n_sm;
  gradient_kernel<<<blocks, 256, 0, c->stream>>>(a, grad, reinterpret_cast<c128*>(dodrho));
  return cuda_status(cudaGetLastError());
}

}  // namespace pngf
