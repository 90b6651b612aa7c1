// Host-side check of the consistency checks on a prepared instance (check_prepared): the
// preprocessing of a valid mesh passes them (in double and with dual numbers), and each of a
// list of planted mistakes in the prepared arrays -- an index out of range, a link that is not
// mutual, a flipped normal, swapped least-squares components, a shifted offset, a wrong area,
// a bad time step -- is caught.  Input: a binary mesh file (nodes, cells, boundary edges,
// periodic pairs).  Prints "<case> <return code> <message>" per line.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <functional>
#include <string>
#include <utility>
#include <vector>

#include "fvlbm_internal.h"

using namespace fvlbm;

template <class T>
static bool read_vec(FILE *f, std::vector<T> &v, size_t n) {
    v.resize(n);
    return n == 0 || fread(v.data(), sizeof(T), n, f) == n;
}

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int nn = 0, nc = 0, nb = 0, npair = 0;
    std::vector<double> xy, bval, shift;
    std::vector<int> cptr, cnodes, bnodes, btype, pairs;
    bool ok = fread(&nn, 4, 1, f) == 1 && read_vec(f, xy, 2 * static_cast<size_t>(nn));
    ok = ok && fread(&nc, 4, 1, f) == 1 && read_vec(f, cptr, nc + 1);
    ok = ok && read_vec(f, cnodes, cptr.empty() ? 0 : cptr.back());
    ok = ok && fread(&nb, 4, 1, f) == 1 && read_vec(f, bnodes, 2 * static_cast<size_t>(nb));
    ok = ok && read_vec(f, btype, nb) && read_vec(f, bval, 5 * static_cast<size_t>(nb));
    ok = ok && fread(&npair, 4, 1, f) == 1 && read_vec(f, pairs, 2 * static_cast<size_t>(npair));
    ok = ok && read_vec(f, shift, 2 * static_cast<size_t>(npair));
    fclose(f);
    if (!ok) return 2;
    fvlbm_mesh M{nn, xy.data(), nc, cptr.data(), cnodes.data()};
    fvlbm_bc B{nb, bnodes.data(), btype.data(), bval.data(), npair, pairs.data(), shift.data()};
    fvlbm_params p{};
    p.nu = 1e-3;
    p.rho0 = 1.0;
    p.cfl = 0.5;
    Prepared P0;
    std::string why;
    int rc = prepare_instance(M, B, p, &P0, &why);
    printf("valid %d %s\n", rc, why.c_str());
    if (rc) return 0;
    {
        std::vector<Dual> xyd(xy.size());
        for (size_t i = 0; i < xy.size(); ++i) xyd[i] = Dual(xy[i], 0.0);
        PreparedT<Dual> D;
        std::string w;
        const int rd = prepare_instance_t<Dual>(M, B, p, xyd.data(), &D, &w);
        printf("valid_dual %d %s\n", rd, w.c_str());
    }
    const size_t np = P0.np;
    // a cell with an interior face (slot mi, neighbour v) and two cells with a boundary face
    int ki = -1, mi = -1, kb = -1, mb = -1, kb2 = -1, mb2 = -1;
    for (int k = 0; k < P0.nc && (ki < 0 || kb2 < 0); ++k)
        for (int m = 0; m < P0.nface[k]; ++m) {
            const int v = P0.nbr[m * np + k];
            if (v >= 0 && ki < 0) { ki = k; mi = m; }
            if (v < 0 && v != kNone) {
                if (kb < 0) { kb = k; mb = m; }
                else if (kb2 < 0 && k != kb) { kb2 = k; mb2 = m; }
            }
        }
    if (ki < 0 || kb2 < 0) return 3;
    const size_t si = static_cast<size_t>(mi) * np + ki, sb = static_cast<size_t>(mb) * np + kb;
    const int v = P0.nbr[si], fb = -(P0.nbr[sb] + 1);
    const int mi1 = (mi + 1) % P0.nface[ki];
    double h = 0.0;
    for (int m = 0; m < P0.nface[ki]; ++m)
        h = std::max(h, std::abs(P0.gq[(2 * m) * np + ki]) + std::abs(P0.gq[(2 * m + 1) * np + ki]));
    std::vector<std::pair<const char *, std::function<void(Prepared &)>>> plants = {
        {"nbr_out_of_range", [&](Prepared &P) { P.nbr[si] = P.nc; }},
        {"back_slot", [&](Prepared &P) { P.back[si] = (P.back[si] + 1) % P.nface[v]; }},
        {"link_not_mutual", [&](Prepared &P) { P.nbr[si] = (v + 1) % P.nc == ki ? (v + 2) % P.nc : (v + 1) % P.nc; }},
        {"open_face", [&](Prepared &P) { P.nbr[si] = kNone; }},
        {"bowner", [&](Prepared &P) { P.bowner[fb] = (P.bowner[fb] + 1) % P.nc; }},
        {"bface_twice", [&](Prepared &P) { P.nbr[static_cast<size_t>(mb2) * np + kb2] = -(fb + 1); }},
        {"padding_face", [&](Prepared &P) { P.nface[P.nc] = 3; }},
        {"padding_slot", [&](Prepared &P) { P.nbr[P.nc] = 0; }},
        {"slot_past_faces", [&](Prepared &P) {
             for (int k = 0; k < P.nc; ++k)
                 if (P.nface[k] == 3) { P.back[3 * np + k] = 0; return; }
             P.nbr[P.nc] = 0;
         }},
        {"perm_duplicate", [&](Prepared &P) { P.perm[1] = P.perm[0]; }},
        {"bedge_order", [&](Prepared &P) { std::swap(P.bedge_of[0], P.bedge_of[1]); }},
        {"btype_periodic", [&](Prepared &P) { P.btype[fb] = FVLBM_BC_PERIODIC; }},
        {"array_size", [&](Prepared &P) { P.lsq.pop_back(); }},
        {"area", [&](Prepared &P) { P.area[ki] *= 1.001; }},
        {"gq_shift", [&](Prepared &P) {
             for (int m = 0; m < P.nface[ki]; ++m) P.gq[(2 * m) * np + ki] += 0.01 * h;
         }},
        {"gq_node_order", [&](Prepared &P) {
             const int nf = P.nface[ki];
             for (int c = 0; c < 2; ++c) {
                 const double first = P.gq[c * np + ki];
                 for (int m = 0; m + 1 < nf; ++m) P.gq[(2 * m + c) * np + ki] = P.gq[(2 * m + 2 + c) * np + ki];
                 P.gq[(2 * (nf - 1) + c) * np + ki] = first;
             }
         }},
        {"sn_sign", [&](Prepared &P) {
             P.sn[(2 * mi) * np + ki] = -P.sn[(2 * mi) * np + ki];
             P.sn[(2 * mi + 1) * np + ki] = -P.sn[(2 * mi + 1) * np + ki];
         }},
        {"sn_slot", [&](Prepared &P) {
             for (int c = 0; c < 2; ++c)
                 std::swap(P.sn[(2 * mi + c) * np + ki], P.sn[(2 * mi1 + c) * np + ki]);
         }},
        {"rown_shift", [&](Prepared &P) { P.rown[(2 * mi) * np + ki] += 0.01 * h; }},
        {"rnbr_own", [&](Prepared &P) {
             for (int c = 0; c < 2; ++c) P.rnbr[(2 * mi + c) * np + ki] = P.rown[(2 * mi + c) * np + ki];
         }},
        {"dvec_not_reversed", [&](Prepared &P) {
             for (int c = 0; c < 2; ++c) P.dvec[(2 * mi + c) * np + ki] *= 1.01;
             P.dinv[static_cast<size_t>(mi) * np + ki] /= 1.01;
         }},
        {"dinv", [&](Prepared &P) { P.dinv[si] *= 1.001; }},
        {"boundary_dvec", [&](Prepared &P) {
             for (int c = 0; c < 2; ++c) P.dvec[(2 * mb + c) * np + kb] *= 1.01;
             P.dinv[sb] /= 1.01;
         }},
        {"lsq_swap", [&](Prepared &P) { std::swap(P.lsq[(2 * mi) * np + ki], P.lsq[(2 * mi + 1) * np + ki]); }},
        {"lsq_dropped_face", [&](Prepared &P) {
             P.lsq[(2 * mi) * np + ki] = 0.0;
             P.lsq[(2 * mi + 1) * np + ki] = 0.0;
         }},
        {"bnrm_sign", [&](Prepared &P) { P.bnrm[2 * fb] = -P.bnrm[2 * fb]; P.bnrm[2 * fb + 1] = -P.bnrm[2 * fb + 1]; }},
        {"blen", [&](Prepared &P) { P.blen[fb] *= 1.001; }},
        {"wdist_nan", [&](Prepared &P) { P.wdist[ki] = std::nan(""); }},
        {"dt_zero", [&](Prepared &P) { P.dt = 0.0; }},
        {"dt_cell_negative", [&](Prepared &P) { P.dt_cell.assign(np, P.dt); P.dt_cell[ki] = -1.0; }},
    };
    for (auto &pl : plants) {
        Prepared P = P0;
        pl.second(P);
        std::string w;
        const int r = check_prepared(P, &w);
        printf("%s %d %s\n", pl.first, r, w.c_str());
    }
    return 0;
}
