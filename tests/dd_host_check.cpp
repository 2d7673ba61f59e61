// Host driver for the double-float arithmetic of dd.cuh: reads operand
// pairs (hi lo) from stdin, one operation per line, and prints the result as
// exact float bit patterns.  Built with floating-point contraction off.
#include <cstdio>
#include <cstring>
#include <cstdint>
#include "dd.cuh"
using namespace pngf;

static unsigned bits(float f) {
  unsigned u;
  std::memcpy(&u, &f, 4);
  return u;
}
static float fl(unsigned u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

int main() {
  char op[16];
  unsigned a0, a1, b0, b1;
  while (std::scanf("%15s %x %x %x %x", op, &a0, &a1, &b0, &b1) == 5) {
    const dd x{fl(a0), fl(a1)}, y{fl(b0), fl(b1)};
    dd z{0.0f, 0.0f};
    if (!std::strcmp(op, "add")) z = dd_add(x, y);
    else if (!std::strcmp(op, "sub")) z = dd_sub(x, y);
    else if (!std::strcmp(op, "mul")) z = dd_mul(x, y);
    else if (!std::strcmp(op, "mulf")) z = dd_mul_f(x, y.hi);
    else if (!std::strcmp(op, "rcp")) z = dd_rcp(x);
    else if (!std::strcmp(op, "sqrt")) z = dd_sqrt(x);
    else if (!std::strcmp(op, "gt")) z = dd{dd_gt(x, y) ? 1.0f : 0.0f, 0.0f};
    std::printf("%08x %08x\n", bits(z.hi), bits(z.lo));
  }
  return 0;
}
