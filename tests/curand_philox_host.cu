// Host-side evaluation of cuRAND's Philox4x32-10 block function, used by the
// oracle tests as an independent library reference.  cuRAND marks the
// function device-only by default; its header also carries a host code path,
// which this program selects by defining the header's QUALIFIERS macro.
// Reads lines "c0 c1 c2 c3 k0 k1" (decimal) from stdin, prints the 4 outputs.
#define QUALIFIERS static inline __host__ __device__
#include <cstdio>
#include <vector_types.h>
#include <curand_philox4x32_x.h>

int main() {
  unsigned c0, c1, c2, c3, k0, k1;
  while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    uint4 c = {c0, c1, c2, c3};
    uint2 k = {k0, k1};
    uint4 r = curand_Philox4x32_10(c, k);
    std::printf("%u %u %u %u\n", r.x, r.y, r.z, r.w);
  }
  return 0;
}
