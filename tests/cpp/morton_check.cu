// Host-only check of the refinement step's Morton keys (meshgen.cu): for the
// block coordinates read from stdin (x y z per line) print the library's key
// and whether decoding it returns the coordinates.  No GPU call.
#include "../../paper_1911_10228_gb300/csrc/meshgen.cu"

#include <cstdio>

int main() {
  long x, y, z;
  while (std::scanf("%ld %ld %ld", &x, &y, &z) == 3) {
    const uint64_t k = flgf::morton_key((int)x, (int)y, (int)z);
    const long dx = (long)flgf::compact3(k >> 2) - (1 << 20), dy = (long)flgf::compact3(k >> 1) - (1 << 20),
               dz = (long)flgf::compact3(k) - (1 << 20);
    std::printf("%llu %d\n", (unsigned long long)k, (int)(dx == x && dy == y && dz == z));
  }
  return 0;
}
