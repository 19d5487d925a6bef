// Test driver (CPU only): assembles the thick-subdomain DSA operator with the library's host setup
// code (sn::dsa_build) on a mesh that exists only on the host, and writes the BSR blocks, so that
// tests can compare the assembled operator with the oracle's without a GPU.
//
// Input (binary, native endianness): int32 dim, nx, ny, nz, p, op, transposed, has_vertices;
// float64 sigma_t[ne], sigma_s[ne]; uint8 mask[ne]; float64 vertices[(nx+1)(ny+1)][2] if 2D and
// has_vertices.  Output: int32 status, nt, n, nnzb; int32 thick[nt], ptr[nt+1], col[nnzb];
// float64 val[nnzb * n * n] (row-major blocks).  status 1 = setup refused (message on stderr).
// With a third argument, the continuous multigrid levels go to that file: int32 count, then per
// level int32 rows, prolongation rows, a_nnz, p_nnz, dense (0/1); CSR a (ptr, col, val), CSR p
// (ptr, col, val; p maps this level to the next finer one), CSR r (the restriction, rows x
// prolongation rows, p_nnz entries) and, for the dense level, its inverse.
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "sn_dsa.h"

namespace {

template <typename T>
bool get(FILE* f, T* dst, size_t count) {
    return std::fread(dst, sizeof(T), count, f) == count;
}

template <typename T>
void put(FILE* f, const T* src, size_t count) {
    if (count) std::fwrite(src, sizeof(T), count, f);
}

}  // namespace

int main(int argc, char** argv) {
    if (argc != 3 && argc != 4) {
        std::fprintf(stderr, "usage: dsa_dump input output [levels]\n");
        return 2;
    }
    FILE* in = std::fopen(argv[1], "rb");
    if (!in) return 2;
    int32_t hdr[8];
    if (!get(in, hdr, 8)) return 2;
    const int dim = hdr[0], nx = hdr[1], ny = hdr[2], nz = dim == 3 ? hdr[3] : 1, p = hdr[4], op = hdr[5];
    const bool transposed = hdr[6] != 0, has_vertices = hdr[7] != 0;
    sn_mesh m;
    m.dim = dim;
    m.p = p;
    m.nx = nx;
    m.ny = ny;
    m.nz = nz;
    const int Q = p + 1;
    m.n = dim == 2 ? Q * Q : Q * Q * Q;
    m.ne = nx * ny * nz;
    m.hx = 1.0 / nx;
    m.hy = 1.0 / ny;
    m.hz = 1.0 / nz;
    m.h_sigma_t.resize(m.ne);
    m.h_sigma_s.resize(m.ne);
    std::vector<unsigned char> mask(m.ne);
    if (!get(in, m.h_sigma_t.data(), m.ne) || !get(in, m.h_sigma_s.data(), m.ne) || !get(in, mask.data(), m.ne))
        return 2;
    if (dim == 2) {  // corner q of element (i, j) is vertex (i + (q & 1), j + (q >> 1)), as sn_mesh_create lays it out
        std::vector<double> V;
        if (has_vertices) {
            V.resize((size_t)(nx + 1) * (ny + 1) * 2);
            if (!get(in, V.data(), V.size())) return 2;
        }
        m.h_corners.resize((size_t)m.ne * 8);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                for (int q = 0; q < 4; ++q) {
                    const int I = i + (q & 1), J = j + (q >> 1);
                    double* c = &m.h_corners[8 * ((size_t)j * nx + i) + 2 * q];
                    c[0] = has_vertices ? V[2 * ((size_t)J * (nx + 1) + I)] : I * m.hx;
                    c[1] = has_vertices ? V[2 * ((size_t)J * (nx + 1) + I) + 1] : J * m.hy;
                }
    }
    std::fclose(in);
    std::string err;
    bool void_conflict = false;
    sn::DsaHierarchy* H = sn::dsa_build(&m, mask.data(), SN_DSA_SIGMA_S, op, transposed, err, &void_conflict);
    FILE* out = std::fopen(argv[2], "wb");
    if (!out) return 2;
    if (!H) {
        std::fprintf(stderr, "%s\n", err.c_str());
        const int32_t res[4] = {1, void_conflict ? 1 : 0, 0, 0};
        put(out, res, 4);
        std::fclose(out);
        return 0;
    }
    const int32_t nnzb = (int32_t)H->l0.col.size();
    const int32_t res[4] = {0, H->nt, H->n, nnzb};
    put(out, res, 4);
    std::vector<int32_t> thick(H->thick.begin(), H->thick.end());
    put(out, thick.data(), thick.size());
    std::vector<int32_t> ptr(H->l0.ptr.begin(), H->l0.ptr.end()), col(H->l0.col.begin(), H->l0.col.end());
    put(out, ptr.data(), ptr.size());
    put(out, col.data(), col.size());
    put(out, H->l0.val.data(), H->l0.val.size());
    std::fclose(out);
    if (argc == 4) {
        FILE* lv = std::fopen(argv[3], "wb");
        if (!lv) return 2;
        const int32_t count = (int32_t)H->levels.size();
        put(lv, &count, 1);
        for (const sn::LevelC& L : H->levels) {
            const int32_t meta[5] = {L.n, (int32_t)L.p_ptr.size() - 1, (int32_t)L.a_val.size(), (int32_t)L.p_val.size(),
                                     L.dense_inv.empty() ? 0 : 1};
            put(lv, meta, 5);
            std::vector<int32_t> ap(L.a_ptr.begin(), L.a_ptr.end()), ac(L.a_col.begin(), L.a_col.end());
            std::vector<int32_t> pp(L.p_ptr.begin(), L.p_ptr.end()), pc(L.p_col.begin(), L.p_col.end());
            put(lv, ap.data(), ap.size());
            put(lv, ac.data(), ac.size());
            put(lv, L.a_val.data(), L.a_val.size());
            put(lv, pp.data(), pp.size());
            put(lv, pc.data(), pc.size());
            put(lv, L.p_val.data(), L.p_val.size());
            std::vector<int32_t> rp(L.r_ptr.begin(), L.r_ptr.end()), rc(L.r_col.begin(), L.r_col.end());
            put(lv, rp.data(), rp.size());
            put(lv, rc.data(), rc.size());
            put(lv, L.r_val.data(), L.r_val.size());
            if (!L.dense_inv.empty()) put(lv, L.dense_inv.data(), L.dense_inv.size());
        }
        std::fclose(lv);
    }
    delete H;  // host-only hierarchy: nothing was uploaded
    return 0;
}
