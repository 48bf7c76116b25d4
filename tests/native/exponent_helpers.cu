// Host-side check of the library's exponent helpers (skf_internal.cuh) against
// the C library: bound_exponent(x) must equal the exponent frexp returns,
// scale_pow2(x, k) must equal ldexp(x, k) bit for bit, and positive_finite
// must hold exactly for finite x > 0.  The same source lines run in the
// kernels (only the bit reinterpretation differs between host and device).
// Prints the number of checked values and mismatches; exits 1 on a mismatch.
#include "../../paper_2208_11447_gb300/csrc/skf_internal.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

using namespace skf;

int main() {
    std::mt19937_64 g(20221130);
    long checked = 0, bad = 0;
    const int ks[] = {-1100, -1075, -1074, -1023, -1022, -600, -60, -52, -1, 0, 1, 52, 500, 1023, 1024};
    auto check = [&](double x) {
        const bool pf = x > 0.0 && std::isfinite(x);
        if (positive_finite(x) != pf) ++bad;
        if (!pf) return;
        int e;
        (void)frexp(x, &e);
        if (bound_exponent(x) != e) ++bad;
        for (int k : ks) {
            const double a = ldexp(x, k), b = scale_pow2(x, k);
            if (memcmp(&a, &b, sizeof a) != 0) ++bad;
        }
        ++checked;
    };
    for (int i = 0; i < 400000; ++i) {   // random bit patterns, both signs
        const unsigned long long b = g();
        double x;
        memcpy(&x, &b, sizeof x);
        check(x);
    }
    for (int i = 0; i < 100000; ++i)     // subnormals and the smallest normals
        check(ldexp((double)(g() >> 11) / 9007199254740992.0, -1022 - (int)(g() % 53)));
    const double special[] = {4.9406564584124654e-324, 2.2250738585072009e-308, 2.2250738585072014e-308, 0.5,
                              0.75, 1.0, 1.7976931348623157e308, 0.0, -0.0, -1.0, INFINITY, -INFINITY, NAN};
    for (double x : special) check(x);
    printf("checked %ld mismatches %ld\n", checked, bad);
    return bad != 0;
}
