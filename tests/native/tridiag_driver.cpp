// Test driver for the host tridiagonal LU with partial pivoting (tridiag_lu):
// reads d and the three diagonals of T from stdin, factorises, solves
// T x = e_j for every j with the factors (the same forward and backward
// substitution the device kernel performs), and prints T^-1 row-major.
#include <cstdio>
#include <vector>

#include "smpm_internal.h"

int main() {
    int d = 0;
    if (std::scanf("%d", &d) != 1 || d < 1) return 2;
    std::vector<double> dl(d - 1), dd(d), du(d - 1), du2;
    std::vector<int> sw;
    for (auto& v : dl) if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : dd) if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : du) if (std::scanf("%lf", &v) != 1) return 2;
    if (!smpm::tridiag_lu(d, dl, dd, du, du2, sw)) { std::printf("singular\n"); return 0; }
    std::vector<double> K((size_t)d * d);
    for (int j = 0; j < d; ++j) {
        std::vector<double> b(d, 0.0);
        b[j] = 1.0;
        for (int i = 0; i + 1 < d; ++i) {
            if (sw[i]) { const double t = b[i]; b[i] = b[i + 1]; b[i + 1] = t - dl[i] * b[i]; }
            else b[i + 1] -= dl[i] * b[i];
        }
        b[d - 1] /= dd[d - 1];
        if (d > 1) b[d - 2] = (b[d - 2] - du[d - 2] * b[d - 1]) / dd[d - 2];
        for (int i = d - 3; i >= 0; --i) b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) / dd[i];
        for (int i = 0; i < d; ++i) K[(size_t)i * d + j] = b[i];
    }
    int swaps = 0;
    for (int s : sw) swaps += s;
    std::printf("swaps %d\n", swaps);
    for (double v : K) std::printf("%.17g\n", v);
    return 0;
}
