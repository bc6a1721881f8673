// Host program for tests/test_philox_split.py: for each line "j p h k0 k1" on
// standard input, prints the four words of philox4x32_10((j, p, h, 0), key)
// and those of its split (philox_head, philox_p1, philox_tail) from the
// library's philox.cuh.  No GPU is used.
#include <cstdio>

#include "philox.cuh"

int main()
{
    unsigned j, p, h, k0, k1;
    while (std::scanf("%u %u %u %u %u", &j, &p, &h, &k0, &k1) == 5) {
        const PhiloxKey key{k0, k1};
        const uint4 d = philox4x32_10(make_uint4(j, p, h, 0u), key);
        const unsigned long long B = (unsigned long long)h * kPhiloxM1;
        const uint4 s = philox_tail(philox_head(j, (uint32_t)B, key), philox_p1(p, (uint32_t)(B >> 32), key), key);
        std::printf("%u %u %u %u %u %u %u %u\n", d.x, d.y, d.z, d.w, s.x, s.y, s.z, s.w);
    }
    return 0;
}
