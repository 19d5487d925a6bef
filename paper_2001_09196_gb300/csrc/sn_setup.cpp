// Host-side setup of libsn: Gauss-Legendre nodal data, the level-symmetric S_N set, and the
// graph helpers of the tiled schedule (CSR construction, strongly connected components).
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "sn_internal.h"

namespace sn {

namespace {

// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double* pn, double* dpn) {
    double p0 = 1.0, p1 = x;
    if (n == 0) {
        *pn = 1.0;
        *dpn = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
    }
    *pn = p1;
    *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

}  // namespace

// Lagrange basis of the nodes g.x (values and derivatives at t).
void lagrange_eval(const GL1D& g, double t, double* val, double* der) {
    const int Q = g.p + 1;
    for (int k = 0; k < Q; ++k) {
        double v = 1.0, d = 0.0;
        for (int m = 0; m < Q; ++m) {
            if (m == k) continue;
            double f = (t - g.x[m]) / (g.x[k] - g.x[m]);
            // product rule: d(v*f) = d*f + v*f'
            d = d * f + v / (g.x[k] - g.x[m]);
            v *= f;
        }
        val[k] = v;
        der[k] = d;
    }
}

GL1D gauss_legendre_nodal(int p) {
    GL1D g;
    g.p = p;
    const int Q = p + 1;
    for (int i = 0; i < Q; ++i) {
        // Newton iteration from the Chebyshev-like initial guess; roots in ascending order
        double x = -std::cos(M_PI * (i + 0.75) / (Q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pn, dpn;
            legendre(Q, x, &pn, &dpn);
            double dx = pn / dpn;
            x -= dx;
            if (std::fabs(dx) < 1e-17) break;
        }
        double pn, dpn;
        legendre(Q, x, &pn, &dpn);
        g.x[i] = x;
        g.w[i] = 2.0 / ((1.0 - x * x) * dpn * dpn);
    }
    double val[kMaxP + 1], der[kMaxP + 1];
    for (int a = 0; a < Q; ++a) {
        lagrange_eval(g, g.x[a], val, der);
        for (int k = 0; k < Q; ++k) g.dm[a][k] = der[k];
    }
    lagrange_eval(g, -1.0, val, der);
    for (int k = 0; k < Q; ++k) {
        g.lm[k] = val[k];
        g.dlm[k] = der[k];
    }
    lagrange_eval(g, 1.0, val, der);
    for (int k = 0; k < Q; ++k) {
        g.lp[k] = val[k];
        g.dlp[k] = der[k];
    }
    return g;
}

// Level-symmetric LQ_N set (Lewis & Miller 1984, ch. 4): cosines mu_i^2 = mu_1^2 + (i-1) 2(1-3mu_1^2)/(N-2),
// one octant's points (mu_i, mu_j, mu_k) with i+j+k = N/2-1 (0-based), permutation classes share a weight,
// weights from exact integration of mu^0 and mu^(2k), k = 2..#classes, over one octant.
bool level_symmetric(int N, int dim, std::vector<double>& dirs, std::vector<double>& wts) {
    double mu1;
    switch (N) {
        case 4: mu1 = 0.3500212; break;
        case 6: mu1 = 0.2666355; break;
        case 8: mu1 = 0.2182179; break;
        default: return false;
    }
    const int n = N / 2;
    std::vector<double> mu(n);
    for (int i = 0; i < n; ++i) mu[i] = std::sqrt(mu1 * mu1 + i * 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2));
    struct Pt { int i, j, k, cls; };
    std::vector<Pt> pts;
    std::vector<std::vector<int>> classes;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n - i; ++j) {
            int k = n - 1 - i - j;
            std::vector<int> key = {i, j, k};
            std::sort(key.begin(), key.end());
            int c = -1;
            for (size_t q = 0; q < classes.size(); ++q)
                if (classes[q] == key) c = (int)q;
            if (c < 0) {
                classes.push_back(key);
                c = (int)classes.size() - 1;
            }
            pts.push_back({i, j, k, c});
        }
    // sort classes lexicographically so the linear system is in a canonical order
    std::vector<int> order(classes.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return classes[a] < classes[b]; });
    std::vector<int> rank(classes.size());
    for (size_t q = 0; q < order.size(); ++q) rank[order[q]] = (int)q;
    const int nc = (int)classes.size();
    std::vector<double> A(nc * nc, 0.0), b(nc, 0.0);
    for (int r = 0; r < nc; ++r) {
        int k = (r == 0) ? 0 : r + 1;  // moments 0, 2, 3, ...
        for (const Pt& p : pts) A[r * nc + rank[p.cls]] += std::pow(mu[p.i], 2 * k);
        b[r] = 1.0 / (2 * k + 1);
    }
    // Gaussian elimination with partial pivoting
    for (int c = 0; c < nc; ++c) {
        int piv = c;
        for (int r = c + 1; r < nc; ++r)
            if (std::fabs(A[r * nc + c]) > std::fabs(A[piv * nc + c])) piv = r;
        for (int q = 0; q < nc; ++q) std::swap(A[c * nc + q], A[piv * nc + q]);
        std::swap(b[c], b[piv]);
        for (int r = c + 1; r < nc; ++r) {
            double f = A[r * nc + c] / A[c * nc + c];
            for (int q = c; q < nc; ++q) A[r * nc + q] -= f * A[c * nc + q];
            b[r] -= f * b[c];
        }
    }
    std::vector<double> wc(nc);
    for (int c = nc - 1; c >= 0; --c) {
        double s = b[c];
        for (int q = c + 1; q < nc; ++q) s -= A[c * nc + q] * wc[q];
        wc[c] = s / A[c * nc + c];
    }
    const int noct = dim == 3 ? 8 : 4;
    dirs.clear();
    wts.clear();
    double total = 0.0;
    for (int o = 0; o < noct; ++o) {
        double sx = (o & 1) ? -1.0 : 1.0, sy = (o & 2) ? -1.0 : 1.0, sz = (o & 4) ? -1.0 : 1.0;
        for (const Pt& p : pts) {
            dirs.push_back(sx * mu[p.i]);
            dirs.push_back(sy * mu[p.j]);
            dirs.push_back(sz * mu[p.k]);
            double w = wc[rank[p.cls]];
            wts.push_back(w);
            total += w;
        }
    }
    for (double& w : wts) w *= kFourPi / total;
    return true;
}

// Strongly connected components of a directed graph in CSR form (iterative Tarjan).
int strong_components(int n, const std::vector<int>& ptr, const std::vector<int>& adj, std::vector<int>& comp) {
    std::vector<int> index(n, -1), low(n, 0), stack;
    std::vector<char> on_stack(n, 0);
    std::vector<std::pair<int, int>> call;  // (vertex, next edge)
    comp.assign(n, -1);
    int counter = 0, n_comp = 0;
    for (int root = 0; root < n; ++root) {
        if (index[root] >= 0) continue;
        index[root] = low[root] = counter++;
        stack.push_back(root);
        on_stack[root] = 1;
        call.push_back({root, ptr[root]});
        while (!call.empty()) {
            const int v = call.back().first;
            if (call.back().second < ptr[v + 1]) {
                const int w = adj[call.back().second++];
                if (index[w] < 0) {
                    index[w] = low[w] = counter++;
                    stack.push_back(w);
                    on_stack[w] = 1;
                    call.push_back({w, ptr[w]});
                } else if (on_stack[w]) {
                    low[v] = std::min(low[v], index[w]);
                }
                continue;
            }
            if (low[v] == index[v]) {
                int w;
                do {
                    w = stack.back();
                    stack.pop_back();
                    on_stack[w] = 0;
                    comp[w] = n_comp;
                } while (w != v);
                ++n_comp;
            }
            call.pop_back();
            if (!call.empty()) low[call.back().first] = std::min(low[call.back().first], low[v]);
        }
    }
    return n_comp;
}

void to_csr(int n, std::vector<std::pair<int, int>>& edges, std::vector<int>& ptr, std::vector<int>& adj) {
    std::sort(edges.begin(), edges.end());
    edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    ptr.assign(n + 1, 0);
    for (const auto& e : edges) ptr[e.first + 1]++;
    for (int i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
    adj.resize(edges.size());
    for (size_t k = 0; k < edges.size(); ++k) adj[k] = edges[k].second;  // sorted by source: CSR order
}

}  // namespace sn
