// Host-side check of the grid split (split_grid in the library's device
// header) against its definition: h = G rint(x / G), l = g rint((x - h) / g),
// g = G 2^-24, rint with ties to even, for random coordinates, exact ties on
// both grids, values far below the grid, zero and subnormals.  Built by
// tests/test_grid_split_cpu.py with nvcc and run on the host.
#include <cfenv>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "../paper_2004_04817_gb300/csrc/rbf_device.cuh"

static void by_definition(double x, double G, float &h, float &l)
{
    const double hd = std::nearbyint(x / G) * G;   // x / G is exact: G is a power of two
    const double g = std::ldexp(G, -24);
    h = (float)hd;
    l = (float)(std::nearbyint((x - hd) / g) * g);
    if (h == 0.0f) h = 0.0f;   // +0 for a zero part
    if (l == 0.0f) l = 0.0f;
}

int main()
{
    std::fesetround(FE_TONEAREST);
    std::mt19937_64 rng(20041);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    long n = 0, bad = 0;
    for (int k = -95; k <= 100; ++k) {
        const double G = std::ldexp(1.0, k - 23), g = std::ldexp(G, -24);
        for (int t = 0; t < 3000; ++t) {
            double x;
            switch (t % 6) {
            case 0: x = U(rng) * std::ldexp(1.0, k) * 0.9999999; break;
            case 1: x = (std::floor(U(rng) * 8e6) + 0.5) * G; break;                       // tie on G
            case 2: x = std::floor(U(rng) * 8e6) * G + (std::floor(U(rng) * 8e6) + 0.5) * g; break;  // tie on g
            case 3: x = U(rng) * std::ldexp(1.0, k - 40); break;
            case 4: x = U(rng) * std::ldexp(1.0, k - 80); break;
            default: x = (std::floor(U(rng) * 8e6) + 0.5) * G + (U(rng) < 0.0 ? -1 : 1) * std::ldexp(g, -30);
            }
            if (!(std::fabs(x) < std::ldexp(1.0, k)))
                continue;
            float h1, l1, h2, l2;
            by_definition(x, G, h1, l1);
            rbf::split_grid(x, G, h2, l2);
            ++n;
            if (std::memcmp(&h1, &h2, 4) != 0 || std::memcmp(&l1, &l2, 4) != 0) {
                if (bad < 5)
                    std::printf("k %d x %a: definition (%a, %a), split_grid (%a, %a)\n", k, x, h1, l1, h2, l2);
                ++bad;
            }
        }
    }
    const double special[] = {0.0, -0.0, 5e-324, -5e-324, 1e-310, -1e-310};
    for (double x : special) {
        float h1, l1, h2, l2;
        by_definition(x, 1.0 / 1024, h1, l1);
        rbf::split_grid(x, 1.0 / 1024, h2, l2);
        ++n;
        if (std::memcmp(&h1, &h2, 4) != 0 || std::memcmp(&l1, &l2, 4) != 0) {
            std::printf("special %a\n", x);
            ++bad;
        }
    }
    std::printf("grid split: %ld cases, %ld mismatches\n", n, bad);
    return bad != 0;
}
