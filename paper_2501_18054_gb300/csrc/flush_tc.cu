// Stand-alone launches of the tensor-core fold (see flush_tc.cuh): a prepare
// pass over the whole grid, then a tile pass of 256-thread CTAs that each own
// 256 tensor-memory columns (two accumulators).  Used by the single-call accept path when the
// delayed set is full; the persistent search runs the same device code.
#include "flush_tc.cuh"

namespace pngf {
namespace {

__global__ void flush_tc_prepare_kernel(SweepArgs a, unsigned char* imgA, unsigned char* imgB) {
  const int r = a.ctl->r_delay;
  if (r < a.R) return;
  tc_prepare(a, r, imgA, imgB, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(256, 1) flush_tc_kernel(SweepArgs a, const unsigned char* imgA,
                                                       const unsigned char* imgB) {
  extern __shared__ __align__(128) unsigned char tc_dyn[];
  __shared__ __align__(8) unsigned long long bars[TC_NBAR];
  __shared__ unsigned tmem_slot;
  const int r = a.ctl->r_delay;
  if (r < a.R) return;
  TcState st{};
  tc_setup(st, bars, &tmem_slot, tc_tmem_cols(2));
  const bool ok = tc_fold_tiles<2>(a, r, imgA, imgB, tc_dyn, st, blockIdx.x, gridDim.x);
  if (!ok && threadIdx.x == 0) latch_status(a.ctl, PNGF_ETIMEOUT);
  tc_teardown(st, !ok);  // after a failure: bounded wait for what was issued
}

}  // namespace

pngf_status flush_tc_launch(pngf_ctx* c) {
  SweepArgs a = make_args(c);
  unsigned char* imgA = reinterpret_cast<unsigned char*>(c->ws) + c->L.tcimg;
  unsigned char* imgB = imgA + c->L.tcimgA_bytes;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(flush_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_fold_smem(2)) != cudaSuccess)
      return PNGF_ECUDA;
    attr = true;
  }
  flush_tc_prepare_kernel<<<c->n_sm * 4, 256, 0, c->stream>>>(a, imgA, imgB);
  flush_tc_kernel<<<c->n_sm, 256, tc_fold_smem(2), c->stream>>>(a, imgA, imgB);
  return cuda_status(cudaGetLastError());
}

}  // namespace pngf
