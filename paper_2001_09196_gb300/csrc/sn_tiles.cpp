// Host-side construction of the tiled sweep schedule (TileSets, sn_internal.h).
//
// The transport update (Sec. 1) solves, per direction, a block lower-triangular system whose
// order is the upwind graph.  The tiled schedule groups the elements of a direction into tasks:
// the elements of every strongly connected component of the tile-level upwind graph (one tile
// in the common case; several where vertex jitter reverses faces on a tile boundary).  The
// component graph is acyclic, so listing tasks by their Kahn level makes every task's upwind
// tasks appear earlier in the list, which is what makes the persistent kernel deadlock free:
// the earliest unfinished task that has been claimed depends only on finished tasks.  Inside a
// task the elements run in increasing global level (the level sets of the mesh), so a CTA only
// has to synchronise itself between levels and to wait for upwind elements of other tasks.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <utility>
#include <vector>

#include "sn_internal.h"

namespace sn {

namespace {

template <typename T>
cudaError_t upload(T** d, const std::vector<T>& h) {
    cudaError_t err = cudaMalloc(d, std::max<size_t>(1, h.size()) * sizeof(T));
    if (err != cudaSuccess) {
        *d = nullptr;
        return err;
    }
    return h.empty() ? cudaSuccess : cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

void free_tiles(sn_mesh* m) {
    TileSets& t = m->tiles;
    if (t.tasks) cudaFree(t.tasks);
    if (t.lvl_ptr) cudaFree(t.lvl_ptr);
    if (t.items) cudaFree(t.items);
    t = TileSets{};
}

cudaError_t build_tiles(sn_mesh* m, int edge, cudaStream_t s) {
    free_tiles(m);
    const int nx = m->nx, ny = m->ny, nz = m->dim == 3 ? m->nz : 1, ne = m->ne, nd = m->nd, nf = 2 * m->dim;
    const long long total = (long long)nd * ne;
    if (total >= INT_MAX || edge < 1) return cudaErrorInvalidValue;
    const std::vector<int>& lev = m->levels.h_level;
    if ((long long)lev.size() != total) return cudaErrorInvalidValue;
    std::vector<unsigned char> mask(total);
    unsigned char* d_mask = nullptr;
    cudaError_t err = cudaMalloc(&d_mask, total);
    if (err != cudaSuccess) return err;
    err = launch_upwind_mask(m, d_mask, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(mask.data(), d_mask, total, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    cudaFree(d_mask);
    if (err != cudaSuccess) return err;

    const int tx = (nx + edge - 1) / edge, ty = (ny + edge - 1) / edge, tz = (nz + edge - 1) / edge;
    const int nt = tx * ty * tz;
    std::vector<int> tile(ne), nbr((size_t)ne * nf, -1);
    for (int e = 0; e < ne; ++e) {
        const int i = e % nx, j = (e / nx) % ny, k = e / (nx * ny);
        tile[e] = i / edge + tx * (j / edge + ty * (k / edge));
        const int c[3] = {i, j, k}, n[3] = {nx, ny, nz};
        for (int f = 0; f < nf; ++f) {
            const int ax = f >> 1, dl = (f & 1) ? 1 : -1;
            int cc[3] = {c[0], c[1], c[2]};
            cc[ax] += dl;
            if (cc[ax] >= 0 && cc[ax] < n[ax]) nbr[(size_t)e * nf + f] = cc[0] + nx * (cc[1] + ny * cc[2]);
        }
    }
    std::vector<int> tptr(nt + 1, 0), telem(ne);
    for (int e = 0; e < ne; ++e) tptr[tile[e] + 1]++;
    for (int t = 0; t < nt; ++t) tptr[t + 1] += tptr[t];
    {
        std::vector<int> fill(tptr.begin(), tptr.end() - 1);
        for (int e = 0; e < ne; ++e) telem[fill[tile[e]]++] = e;
    }

    struct TaskRec {
        int klev, minlev, d, first, lvl_first, n_lev;
    };
    std::vector<TaskRec> recs;
    std::vector<int> h_lvl;
    std::vector<int2> h_items;
    h_items.reserve(total);
    int max_run = 0;
    std::vector<std::pair<int, int>> edges;
    std::vector<int> ptr, adj, comp, cptr, cadj, indeg, klev, order, elems;
    for (int d = 0; d < nd; ++d) {
        const unsigned char* mk = mask.data() + (size_t)d * ne;
        const int* lv = lev.data() + (size_t)d * ne;
        edges.clear();
        for (int e = 0; e < ne; ++e)
            for (int f = 0; f < nf; ++f)
                if ((mk[e] >> f) & 1) {
                    const int u = nbr[(size_t)e * nf + f];
                    if (tile[u] != tile[e]) edges.push_back({tile[u], tile[e]});
                }
        to_csr(nt, edges, ptr, adj);
        const int nc = strong_components(nt, ptr, adj, comp);
        // component graph and its Kahn levels
        edges.clear();
        for (int a = 0; a < nt; ++a)
            for (int q = ptr[a]; q < ptr[a + 1]; ++q)
                if (comp[a] != comp[adj[q]]) edges.push_back({comp[a], comp[adj[q]]});
        to_csr(nc, edges, cptr, cadj);
        indeg.assign(nc, 0);
        for (int v : cadj) indeg[v]++;
        klev.assign(nc, 0);
        order.clear();
        for (int c = 0; c < nc; ++c)
            if (!indeg[c]) order.push_back(c);
        for (size_t q = 0; q < order.size(); ++q) {
            const int c = order[q];
            for (int k = cptr[c]; k < cptr[c + 1]; ++k) {
                const int v = cadj[k];
                klev[v] = std::max(klev[v], klev[c] + 1);
                if (--indeg[v] == 0) order.push_back(v);
            }
        }
        if ((int)order.size() != nc) return cudaErrorInvalidValue;  // cannot happen: components form a DAG
        // tiles of every component
        std::vector<std::vector<int>> ctiles(nc);
        for (int t = 0; t < nt; ++t) ctiles[comp[t]].push_back(t);
        for (int c = 0; c < nc; ++c) {
            elems.clear();
            for (int t : ctiles[c]) elems.insert(elems.end(), telem.begin() + tptr[t], telem.begin() + tptr[t + 1]);
            if (elems.empty()) continue;
            std::sort(elems.begin(), elems.end(), [&](int x, int y) { return lv[x] != lv[y] ? lv[x] < lv[y] : x < y; });
            TaskRec rec{klev[c], lv[elems[0]], d, (int)h_items.size(), (int)h_lvl.size(), 0};
            int prev = -1, run = 0;
            for (int e : elems) {
                if (lv[e] != prev) {
                    h_lvl.push_back((int)h_items.size());
                    ++rec.n_lev;
                    prev = lv[e];
                    run = 0;
                }
                max_run = std::max(max_run, ++run);
                int flags = 0;
                for (int f = 0; f < nf; ++f) {
                    const int u = nbr[(size_t)e * nf + f];
                    if (u < 0 || comp[tile[u]] == c) continue;
                    if ((mk[e] >> f) & 1) flags |= 1 << f;                      // u is upwind of e
                    if ((mk[u] >> (f ^ 1)) & 1) flags |= kTilePublish;          // e is upwind of u
                }
                h_items.push_back(make_int2(e, flags));
            }
            h_lvl.push_back((int)h_items.size());
            recs.push_back(rec);
        }
    }
    // claim order: topological within every direction (Kahn level), early wavefronts first
    std::sort(recs.begin(), recs.end(), [](const TaskRec& x, const TaskRec& y) {
        if (x.klev != y.klev) return x.klev < y.klev;
        if (x.minlev != y.minlev) return x.minlev < y.minlev;
        return x.d < y.d;
    });
    std::vector<int4> h_tasks(recs.size());
    for (size_t q = 0; q < recs.size(); ++q) {
        // lvl_first indexes the boundary array; a task with n_lev levels owns n_lev + 1 entries
        h_tasks[q] = make_int4(recs[q].d, recs[q].first, recs[q].lvl_first, recs[q].n_lev);
    }
    TileSets& T = m->tiles;
    if ((err = upload(&T.tasks, h_tasks)) != cudaSuccess || (err = upload(&T.lvl_ptr, h_lvl)) != cudaSuccess ||
        (err = upload(&T.items, h_items)) != cudaSuccess) {
        free_tiles(m);
        return err;
    }
    T.n_tasks = (long long)h_tasks.size();
    T.max_level_items = max_run;
    T.edge = edge;
    return cudaSuccess;
}

}  // namespace sn
