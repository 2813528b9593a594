// Host-side evaluation of cuRAND's Philox4x32-10 block function, used by the
// oracle tests as an independent known-answer source for the oracle's own
// Philox.  The cuRAND header defines the block function for host and device;
// here it is instantiated for the host only and called on counters/keys read
// from stdin, one "c0 c1 c2 c3 k0 k1" line each; it prints the four output words.
#define QUALIFIERS static inline __host__ __device__
#include <cstdio>
#include <curand_philox4x32_x.h>

int main() {
    unsigned c0, c1, c2, c3, k0, k1;
    while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
        uint4 c = make_uint4(c0, c1, c2, c3);
        uint2 k = make_uint2(k0, k1);
        uint4 r = curand_Philox4x32_10(c, k);
        std::printf("%u %u %u %u\n", r.x, r.y, r.z, r.w);
    }
    return 0;
}
