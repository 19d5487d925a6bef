// Test driver (CPU only): runs the library's directed-graph helpers of the tiled schedule on a
// graph read from standard input, so that tests can check them without a GPU.
//   input:  n m, then m lines "source target" (0-based; duplicates allowed)
//   output: the CSR arrays (line "ptr ...", line "adj ..."), then "ncomp K" and one line
//           "comp c_0 ... c_{n-1}" with every vertex's strongly connected component
#include <cstdio>
#include <utility>
#include <vector>

#include "sn_internal.h"

int main() {
    int n = 0, m = 0;
    if (std::scanf("%d %d", &n, &m) != 2 || n < 0 || m < 0) return 2;
    std::vector<std::pair<int, int>> edges;
    for (int k = 0; k < m; ++k) {
        int a = 0, b = 0;
        if (std::scanf("%d %d", &a, &b) != 2 || a < 0 || a >= n || b < 0 || b >= n) return 2;
        edges.push_back({a, b});
    }
    std::vector<int> ptr, adj, comp;
    sn::to_csr(n, edges, ptr, adj);
    const int nc = sn::strong_components(n, ptr, adj, comp);
    std::printf("ptr");
    for (int v : ptr) std::printf(" %d", v);
    std::printf("\nadj");
    for (int v : adj) std::printf(" %d", v);
    std::printf("\nncomp %d\ncomp", nc);
    for (int v : comp) std::printf(" %d", v);
    std::printf("\n");
    return 0;
}
