// Test driver (CPU only): writes the library's quadrature data from its host setup code, so that
// tests can compare it with the oracle and with textbook values without a GPU.
//   quad_dump ls N dim   -> per direction: x y z w (level-symmetric S_N set, weights sum to 4 pi)
//   quad_dump gl p       -> per node: x w l(-1) l(+1) and the row of derivatives l_k'(x_a)
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "sn_internal.h"

int main(int argc, char** argv) {
    if (argc == 4 && std::strcmp(argv[1], "ls") == 0) {
        std::vector<double> dirs, wts;
        if (!sn::level_symmetric(std::atoi(argv[2]), std::atoi(argv[3]), dirs, wts)) return 1;
        for (size_t d = 0; d < wts.size(); ++d)
            std::printf("%.17g %.17g %.17g %.17g\n", dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2], wts[d]);
        return 0;
    }
    if (argc == 3 && std::strcmp(argv[1], "gl") == 0) {
        const int p = std::atoi(argv[2]);
        if (p < 1 || p > sn::kMaxP) return 1;
        const sn::GL1D g = sn::gauss_legendre_nodal(p);
        for (int a = 0; a <= p; ++a) {
            std::printf("%.17g %.17g %.17g %.17g", g.x[a], g.w[a], g.lm[a], g.lp[a]);
            for (int k = 0; k <= p; ++k) std::printf(" %.17g", g.dm[a][k]);
            std::printf("\n");
        }
        return 0;
    }
    std::fprintf(stderr, "usage: quad_dump ls N dim | quad_dump gl p\n");
    return 2;
}
