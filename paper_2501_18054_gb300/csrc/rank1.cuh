// Kept-flip update of the FP64 maintained inverse, W += alpha c c^T (Eq. 9 in
// field form; complex symmetric W, upper triangle), with the scaled column
// ac = alpha c formed once per kept flip.  Used by the persistent FP64 search
// and the batch kernel; one complex FMA per element of the triangle.
#pragma once

#include "sweep_common.cuh"

namespace pngf {
namespace {

// c_j = W[k][j] (j >= k) or W[j][k] (j < k) into a.cbuf, and ac_j = alpha c_j,
// for j in [pb, pe)
__device__ void gather_column_ac(const SweepArgs& a, int k, c128 alpha, c128* ac, int pb, int pe) {
  for (int j = pb + threadIdx.x; j < pe; j += blockDim.x) {
    const c128 cj = (j >= k) ? a.W[(size_t)k * a.ldw + j] : a.W[(size_t)j * a.ldw + k];
    a.cbuf[j] = cj;
    ac[j] = cmul(alpha, cj);
  }
}

// W[i][j] += ac_i c_j on packed elements [eb, ee) of the upper triangle.
// Thread t walks elements eb + t + m*blockDim; four consecutive steps of the
// walk are issued together so that four independent loads are in flight.
// (Forming alpha c_i per element instead costs a complex product per element
// on the FP64 pipe, whose instructions cost a full issue slot even where only
// some lanes change row.)
__device__ void rank1_upper_ac(c128* __restrict__ W, int n, int ldw, const c128* __restrict__ ac,
                               const c128* __restrict__ c, long long eb, long long ee) {
  long long e = eb + threadIdx.x;
  if (e >= ee) return;
  const int stride = blockDim.x;
  int i0, j0;
  tri_rc(e, n, i0, j0);
  while (e + 3LL * stride < ee) {
    int i1 = i0, j1 = j0;
    tri_step(i1, j1, n, stride);
    int i2 = i1, j2 = j1;
    tri_step(i2, j2, n, stride);
    int i3 = i2, j3 = j2;
    tri_step(i3, j3, n, stride);
    c128* p0 = W + (size_t)i0 * ldw + j0;
    c128* p1 = W + (size_t)i1 * ldw + j1;
    c128* p2 = W + (size_t)i2 * ldw + j2;
    c128* p3 = W + (size_t)i3 * ldw + j3;
    const c128 w0 = *p0, w1 = *p1, w2 = *p2, w3 = *p3;
    const c128 c0 = c[j0], c1 = c[j1], c2 = c[j2], c3 = c[j3];
    const c128 a0 = ac[i0], a1 = ac[i1], a2 = ac[i2], a3 = ac[i3];
    *p0 = cfma(a0, c0, w0);
    *p1 = cfma(a1, c1, w1);
    *p2 = cfma(a2, c2, w2);
    *p3 = cfma(a3, c3, w3);
    i0 = i3;
    j0 = j3;
    tri_step(i0, j0, n, stride);
    e += 4LL * stride;
  }
  for (; e < ee; e += stride) {
    c128* p = W + (size_t)i0 * ldw + j0;
    *p = cfma(ac[i0], c[j0], *p);
    tri_step(i0, j0, n, stride);
  }
}

}  // namespace
}  // namespace pngf
