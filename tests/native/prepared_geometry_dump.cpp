// Dumps, in input cell order, what the library's host preprocessing gives the kernels for one
// mesh: the cell area, the wall distance, the time step (CFL 0.5) and the least-squares
// gradient of a given cell field with given boundary-edge values.  The gradient is formed as
// the kernels form it: sum over face slots of W_m (phi_neighbour - phi_i), with the boundary
// face value for a boundary slot.  Input: the binary mesh file of prepared_check.cpp followed
// by phi [n_cells] and phi_b [n_bedges].  A third argument "local" asks for local time
// stepping.  Output: a binary file of doubles, dt, then per input cell (area, wall distance,
// gx, gy, the cell's own time step).
#include <cstdio>
#include <string>
#include <vector>

#include "fvlbm_internal.h"

using namespace fvlbm;

template <class T>
static bool read_vec(FILE *f, std::vector<T> &v, size_t n) {
    v.resize(n);
    return n == 0 || fread(v.data(), sizeof(T), n, f) == n;
}

int main(int argc, char **argv) {
    if (argc < 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int nn = 0, nc = 0, nb = 0, npair = 0;
    std::vector<double> xy, bval, shift, phi, phib;
    std::vector<int> cptr, cnodes, bnodes, btype, pairs;
    bool ok = fread(&nn, 4, 1, f) == 1 && read_vec(f, xy, 2 * static_cast<size_t>(nn));
    ok = ok && fread(&nc, 4, 1, f) == 1 && read_vec(f, cptr, nc + 1);
    ok = ok && read_vec(f, cnodes, cptr.empty() ? 0 : cptr.back());
    ok = ok && fread(&nb, 4, 1, f) == 1 && read_vec(f, bnodes, 2 * static_cast<size_t>(nb));
    ok = ok && read_vec(f, btype, nb) && read_vec(f, bval, 5 * static_cast<size_t>(nb));
    ok = ok && fread(&npair, 4, 1, f) == 1 && read_vec(f, pairs, 2 * static_cast<size_t>(npair));
    ok = ok && read_vec(f, shift, 2 * static_cast<size_t>(npair));
    ok = ok && read_vec(f, phi, nc) && read_vec(f, phib, nb);
    fclose(f);
    if (!ok) return 2;
    fvlbm_mesh M{nn, xy.data(), nc, cptr.data(), cnodes.data()};
    fvlbm_bc B{nb, bnodes.data(), btype.data(), bval.data(), npair, pairs.data(), shift.data()};
    fvlbm_params p{};
    p.nu = 1e-3;
    p.rho0 = 1.0;
    p.cfl = 0.5;
    p.local_dt = argc > 3 && std::string(argv[3]) == "local";
    Prepared P;
    std::string why;
    if (prepare_instance(M, B, p, &P, &why)) {
        fprintf(stderr, "%s\n", why.c_str());
        return 3;
    }
    const size_t np = P.np;
    std::vector<double> out(1 + 5 * static_cast<size_t>(nc));
    out[0] = P.dt;
    for (int k = 0; k < P.nc; ++k) {
        const int i = P.perm[k];
        double gx = 0.0, gy = 0.0;
        for (int m = 0; m < P.nface[k]; ++m) {
            const int v = P.nbr[m * np + k];
            const double q = v >= 0 ? phi[P.perm[v]] : phib[P.bedge_of[-v - 1]];
            gx += P.lsq[(2 * m) * np + k] * (q - phi[i]);
            gy += P.lsq[(2 * m + 1) * np + k] * (q - phi[i]);
        }
        double *row = &out[1 + 5 * static_cast<size_t>(i)];
        row[0] = P.area[k];
        row[1] = P.wdist[k];
        row[2] = gx;
        row[3] = gy;
        row[4] = P.dt_cell.empty() ? P.dt : P.dt_cell[k];
    }
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 2;
    const bool w = fwrite(out.data(), sizeof(double), out.size(), o) == out.size();
    fclose(o);
    return w ? 0 : 2;
}
