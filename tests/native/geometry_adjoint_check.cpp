// Host-side check of the reverse-mode geometry (geometry_adjoint) used by the shape gradient of
// the adjoint: for random adjoints A of the geometry arrays (face normals and lengths, offsets,
// least-squares weights, 1 / |d|, wall distance, cell area, wall normals and lengths) and a random node
// displacement v,
//   <A, d(geometry)/d(xy) v>  from prepare_instance_t<Dual> (forward mode, one direction)
// must equal
//   <geometry_adjoint(A), v>  (reverse mode).
// Reads the mesh file of dual_geometry_check (without its trailing node record) followed by one
// 64-bit seed; prints "forward <value>" and "reverse <value>".
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "fvlbm_internal.h"

using namespace fvlbm;

template <class V>
static bool get(FILE *f, V *p, size_t n) { return fread(p, sizeof(V), n, f) == n; }

// splitmix64 mapped to [-1, 1)
static double uniform(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return static_cast<double>(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int nn = 0, nc = 0, nbe = 0;
    uint64_t seed = 0;
    bool ok = get(f, &nn, 1);
    std::vector<double> xy(2 * static_cast<size_t>(nn));
    ok = ok && get(f, xy.data(), xy.size()) && get(f, &nc, 1);
    std::vector<int> ptr(nc + 1);
    ok = ok && get(f, ptr.data(), ptr.size());
    std::vector<int> cn(ptr[nc]);
    ok = ok && get(f, cn.data(), cn.size()) && get(f, &nbe, 1);
    std::vector<int> bn(2 * static_cast<size_t>(nbe)), bt(nbe);
    std::vector<double> bv(5 * static_cast<size_t>(nbe));
    ok = ok && get(f, bn.data(), bn.size()) && get(f, bt.data(), bt.size()) && get(f, bv.data(), bv.size());
    ok = ok && get(f, &seed, 1);
    fclose(f);
    if (!ok) return 3;
    fvlbm_mesh M{nn, xy.data(), nc, ptr.data(), cn.data()};
    fvlbm_bc B{nbe, bn.data(), bt.data(), bv.data(), 0, nullptr, nullptr};
    fvlbm_params p{};
    p.nu = 1e-3;
    p.rho0 = 1.0;
    p.dt = 1e-3;
    uint64_t s = seed;
    GeometryAdjoint A;
    for (auto *v : {&A.sn, &A.lsq, &A.rown, &A.rnbr}) {
        v->resize(8 * static_cast<size_t>(nc));
        for (double &x : *v) x = uniform(s);
    }
    A.dinv.resize(4 * static_cast<size_t>(nc));
    for (double &x : A.dinv) x = uniform(s);
    A.wdist.resize(nc);
    for (double &x : A.wdist) x = uniform(s);
    A.area.resize(nc);
    for (double &x : A.area) x = uniform(s);
    A.bnrm.resize(2 * static_cast<size_t>(nbe));
    A.blen.resize(nbe);
    for (double &x : A.bnrm) x = uniform(s);
    for (double &x : A.blen) x = uniform(s);
    std::vector<double> dir(xy.size());
    for (double &x : dir) x = 1e-3 * uniform(s);
    // forward mode along dir
    std::vector<Dual> xd(xy.size());
    for (size_t k = 0; k < xy.size(); ++k) xd[k] = Dual(xy[k], dir[k]);
    PreparedT<Dual> D;
    std::string why;
    if (prepare_instance_t<Dual>(M, B, p, xd.data(), &D, &why)) return 4;
    const size_t np = D.np;
    double fwd = 0.0;
    for (int k = 0; k < D.nc; ++k) {
        const size_t i = D.perm[k];
        fwd += A.wdist[i] * D.wdist[k].d + A.area[i] * D.area[k].d;
        for (int l = 0; l < D.nface[k]; ++l) fwd += A.dinv[4 * i + l] * D.dinv[l * np + k].d;
        for (int l = 0; l < D.nface[k]; ++l)
            for (int c = 0; c < 2; ++c) {
                const size_t o = (4 * i + l) * 2 + c, q = (2 * l + c) * np + k;
                fwd += A.sn[o] * D.sn[q].d + A.lsq[o] * D.lsq[q].d + A.rown[o] * D.rown[q].d +
                       A.rnbr[o] * D.rnbr[q].d;
            }
    }
    for (int b = 0; b < D.nb; ++b) {
        const int e = D.bedge_of[b];
        fwd += A.bnrm[2 * e] * D.bnrm[2 * b].d + A.bnrm[2 * e + 1] * D.bnrm[2 * b + 1].d + A.blen[e] * D.blen[b].d;
    }
    // reverse mode
    std::vector<double> g(xy.size());
    if (geometry_adjoint(M, B, A, g.data(), &why)) return 5;
    double rev = 0.0;
    for (size_t k = 0; k < g.size(); ++k) rev += g[k] * dir[k];
    printf("forward %.17g\nreverse %.17g\n", fwd, rev);
    return 0;
}
