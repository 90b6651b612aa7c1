// Host-side check of the dual-number geometry used by the tangent path: derivatives of the
// preprocessed geometry (areas, normals, least-squares weights, face offsets, wall distance)
// with respect to one node's position, from prepare_instance_t<Dual>, against central
// differences of prepare_instance_t<double>.  Reads a mesh from a binary file written by the
// test (layout below) and prints one line per array: name, |FD|, |dual - FD|.
//   int n_nodes; double xy[2 n_nodes]; int n_cells; int cell_ptr[n_cells + 1];
//   int cell_nodes[cell_ptr[n_cells]]; int n_bedges; int bedge_nodes[2 n_bedges];
//   int bedge_type[n_bedges]; double bedge_val[5 n_bedges]; int node; double dx, dy, h
#include <cmath>
#include <cstdio>
#include <vector>

#include "fvlbm_internal.h"

using namespace fvlbm;

template <class V>
static bool get(FILE *f, V *p, size_t n) { return fread(p, sizeof(V), n, f) == n; }

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int nn = 0, nc = 0, nbe = 0, node = 0;
    double dx = 0, dy = 0, h = 0;
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
    ok = ok && get(f, &node, 1) && get(f, &dx, 1) && get(f, &dy, 1) && get(f, &h, 1);
    fclose(f);
    if (!ok) return 3;
    fvlbm_mesh M{nn, xy.data(), nc, ptr.data(), cn.data()};
    fvlbm_bc B{nbe, bn.data(), bt.data(), bv.data(), 0, nullptr, nullptr};
    fvlbm_params p{};
    p.nu = 1e-3;
    p.rho0 = 1.0;
    p.dt = 1e-3;
    std::vector<Dual> xd(xy.size());
    for (size_t k = 0; k < xy.size(); ++k) xd[k] = Dual(xy[k], 0.0);
    xd[2 * node].d = dx;
    xd[2 * node + 1].d = dy;
    PreparedT<Dual> D;
    std::string why;
    if (prepare_instance_t<Dual>(M, B, p, xd.data(), &D, &why)) return 4;
    std::vector<double> xp(xy), xm(xy);
    xp[2 * node] += h * dx; xp[2 * node + 1] += h * dy;
    xm[2 * node] -= h * dx; xm[2 * node + 1] -= h * dy;
    Prepared Pp, Pm;
    M.xy = xp.data();
    if (prepare_instance_t<double>(M, B, p, xp.data(), &Pp, &why)) return 5;
    M.xy = xm.data();
    if (prepare_instance_t<double>(M, B, p, xm.data(), &Pm, &why)) return 6;
    if (Pp.perm != D.perm || Pm.perm != D.perm) return 7;
    auto cmp = [&](const char *name, const std::vector<Dual> &d, const std::vector<double> &a,
                   const std::vector<double> &b) {
        double num = 0, den = 0;
        for (size_t k = 0; k < d.size(); ++k) {
            const double fd = (a[k] - b[k]) / (2 * h);
            num += (d[k].d - fd) * (d[k].d - fd);
            den += fd * fd;
        }
        printf("%s %.17g %.17g\n", name, std::sqrt(den), std::sqrt(num));
    };
    cmp("sn", D.sn, Pp.sn, Pm.sn);
    cmp("lsq", D.lsq, Pp.lsq, Pm.lsq);
    cmp("rown", D.rown, Pp.rown, Pm.rown);
    cmp("rnbr", D.rnbr, Pp.rnbr, Pm.rnbr);
    cmp("dinv", D.dinv, Pp.dinv, Pm.dinv);
    cmp("area", D.area, Pp.area, Pm.area);
    cmp("wdist", D.wdist, Pp.wdist, Pm.wdist);
    cmp("bnrm", D.bnrm, Pp.bnrm, Pm.bnrm);
    cmp("blen", D.blen, Pp.blen, Pm.blen);
    return 0;
}
