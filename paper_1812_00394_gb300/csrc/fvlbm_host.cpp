// fvlbm_host.cpp -- host preprocessing of one solver instance: mesh validation, face
// connectivity, finite-volume geometry (Eq. (advection) needs A, n and Delta l per face), the
// least-squares gradient weights (Step 2 of Sec. 3.2), periodic gluing, wall distance d
// (Sec. 2, needed by f1 and f2), the time step from a CFL number, and a renumbering of
// the cells into compact blocks (Hilbert-seeded breadth-first growth) so that face neighbours
// sit close in memory on the GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "fvlbm_internal.h"

namespace fvlbm {
namespace {

struct Side {
    int cell = -1, local = -1;
};

inline uint64_t edge_id(int a, int b) {
    uint32_t lo = static_cast<uint32_t>(std::min(a, b)), hi = static_cast<uint32_t>(std::max(a, b));
    return (static_cast<uint64_t>(lo) << 32) | hi;
}

// Position of (x, y) along a Hilbert curve over a 2^32 x 2^32 grid (iterative quadrant
// descent with the curve's reflections).  Consecutive keys are face neighbours on the grid, so
// runs of consecutive cells are compact patches with short perimeters.
inline uint64_t hilbert_key(uint64_t x, uint64_t y) {
    uint64_t d = 0;
    for (uint64_t s = uint64_t(1) << 31; s > 0; s >>= 1) {
        const uint64_t rx = (x & s) ? 1 : 0, ry = (y & s) ? 1 : 0;
        d += s * s * ((3 * rx) ^ ry);
        if (ry == 0) {  // rotate / reflect the sub-square
            if (rx == 1) {
                x = (s - 1) - (x & (s - 1)) + (x & ~(s - 1));
                y = (s - 1) - (y & (s - 1)) + (y & ~(s - 1));
            }
            std::swap(x, y);
        }
    }
    return d;
}

template <class S>
S point_segment(S px, S py, S ax, S ay, S bx, S by) {
    const S ex = bx - ax, ey = by - ay;
    const S L2 = ex * ex + ey * ey;
    S t = L2 > S(0.0) ? ((px - ax) * ex + (py - ay) * ey) / L2 : S(0.0);
    t = smin(S(1.0), smax(S(0.0), t));
    const S dx = ax + t * ex - px, dy = ay + t * ey - py;
    return sqrt(dx * dx + dy * dy);
}

template <class S>
struct FaceGeo {
    int nbr = kNone;        // neighbour input cell id, or -(b+1) boundary edge, or kNone
    int back = -1;          // local slot of this face in the neighbour's face list
    S nx = 0, ny = 0;       // unit outward normal
    S len = 0;
    S xm = 0, ym = 0;
    double sx = 0, sy = 0;  // neighbour centroid offset (periodic shift as seen from here)
};

}  // namespace

template <class S>
int prepare_instance_t(const fvlbm_mesh &m, const fvlbm_bc &bc, const fvlbm_params &p, const S *xy,
                       PreparedT<S> *out, std::string *why) {
    const int nc = m.n_cells;
    if (nc <= 0 || m.n_nodes <= 0 || !m.xy || !m.cell_ptr || !m.cell_nodes) {
        *why = "empty mesh";
        return FVLBM_ERR_BAD_MESH;
    }
    if (!(p.nu > 0.0) || !(p.rho0 > 0.0) || (p.dt <= 0.0 && !(p.cfl > 0.0))) {
        *why = "need nu > 0, rho0 > 0 and dt > 0 or cfl > 0";
        return FVLBM_ERR_BAD_PARAM;
    }
    if (p.local_dt && !(p.cfl > 0.0)) {
        *why = "local time stepping needs cfl > 0";
        return FVLBM_ERR_BAD_PARAM;
    }
    if (!xy) {
        *why = "empty mesh";
        return FVLBM_ERR_BAD_MESH;
    }
    std::vector<S> cx(nc), cy(nc), area(nc);
    std::vector<FaceGeo<S>> face(static_cast<size_t>(nc) * 4);
    std::unordered_map<uint64_t, Side> open;
    open.reserve(static_cast<size_t>(nc) * 3);
    for (int i = 0; i < nc; ++i) {
        const int p0 = m.cell_ptr[i], nv = m.cell_ptr[i + 1] - p0;
        if (nv < 3 || nv > 4) {
            *why = "cell " + std::to_string(i) + " has " + std::to_string(nv) + " nodes";
            return FVLBM_ERR_BAD_MESH;
        }
        for (int l = 0; l < nv; ++l) {
            const int a = m.cell_nodes[p0 + l];
            if (a < 0 || a >= m.n_nodes) {
                *why = "node id out of range";
                return FVLBM_ERR_BAD_MESH;
            }
        }
        // polygon area and centroid, relative to node 0 of the cell for accuracy on small cells
        const int n0 = m.cell_nodes[p0];
        const S ox = xy[2 * n0], oy = xy[2 * n0 + 1];
        S a2 = 0, mx = 0, my = 0;
        for (int l = 0; l < nv; ++l) {
            const int a = m.cell_nodes[p0 + l], b = m.cell_nodes[p0 + (l + 1) % nv];
            const S x0 = xy[2 * a] - ox, y0 = xy[2 * a + 1] - oy;
            const S x1 = xy[2 * b] - ox, y1 = xy[2 * b + 1] - oy;
            const S c = x0 * y1 - x1 * y0;
            a2 += c;
            mx += (x0 + x1) * c;
            my += (y0 + y1) * c;
        }
        if (!(a2 > S(0.0))) {
            *why = "cell " + std::to_string(i) + " has non-positive area (nodes must be CCW)";
            return FVLBM_ERR_BAD_MESH;
        }
        area[i] = S(0.5) * a2;
        cx[i] = ox + mx / (S(3.0) * a2);
        cy[i] = oy + my / (S(3.0) * a2);
        for (int l = 0; l < nv; ++l) {
            const int a = m.cell_nodes[p0 + l], b = m.cell_nodes[p0 + (l + 1) % nv];
            const S ex = xy[2 * b] - xy[2 * a], ey = xy[2 * b + 1] - xy[2 * a + 1];
            FaceGeo<S> &F = face[4 * static_cast<size_t>(i) + l];
            F.len = sqrt(ex * ex + ey * ey);
            F.nx = ey / F.len;
            F.ny = -ex / F.len;
            F.xm = S(0.5) * (xy[2 * a] + xy[2 * b]);
            F.ym = S(0.5) * (xy[2 * a + 1] + xy[2 * b + 1]);
            const uint64_t id = edge_id(a, b);
            auto it = open.find(id);
            if (it == open.end()) {
                open.emplace(id, Side{i, l});
            } else {
                if (it->second.cell < 0) {
                    *why = "edge shared by more than two cells";
                    return FVLBM_ERR_BAD_MESH;
                }
                FaceGeo<S> &G = face[4 * static_cast<size_t>(it->second.cell) + it->second.local];
                F.nbr = it->second.cell;
                F.back = it->second.local;
                G.nbr = i;
                G.back = l;
                it->second.cell = -1;  // closed
            }
        }
    }
    // boundary edges
    const int nbe = bc.n_bedges;
    std::vector<Side> bside(nbe);
    for (int b = 0; b < nbe; ++b) {
        const int a0 = bc.bedge_nodes[2 * b], a1 = bc.bedge_nodes[2 * b + 1];
        auto it = open.find(edge_id(a0, a1));
        if (it == open.end() || it->second.cell < 0) {
            *why = "boundary edge " + std::to_string(b) + " is not a boundary edge of the mesh";
            return FVLBM_ERR_BAD_BC;
        }
        const int t = bc.bedge_type[b];
        if (t < FVLBM_BC_WALL || t > FVLBM_BC_PERIODIC) {
            *why = "unknown boundary type";
            return FVLBM_ERR_BAD_BC;
        }
        bside[b] = it->second;
        face[4 * static_cast<size_t>(it->second.cell) + it->second.local].nbr = -(b + 1);
    }
    std::vector<char> glued(nbe, 0);
    double gap = 0.0;  // largest mismatch of a glued pair (side B's own edge against side A's)
    for (int q = 0; q < bc.n_periodic; ++q) {
        const int ea = bc.periodic_pairs[2 * q], eb = bc.periodic_pairs[2 * q + 1];
        if (ea < 0 || eb < 0 || ea >= nbe || eb >= nbe || glued[ea] || glued[eb]) {
            *why = "bad periodic pair";
            return FVLBM_ERR_BAD_BC;
        }
        const double sx = bc.periodic_shift[2 * q], sy = bc.periodic_shift[2 * q + 1];
        FaceGeo<S> &A = face[4 * static_cast<size_t>(bside[ea].cell) + bside[ea].local];
        FaceGeo<S> &B = face[4 * static_cast<size_t>(bside[eb].cell) + bside[eb].local];
        // edge b must be edge a moved by the shift (traversed the other way by its cell): same
        // length, opposite normals, midpoints one shift apart
        const double la = value_of(A.len), lb = value_of(B.len);
        const double ex = value_of(B.xm) - sx - value_of(A.xm), ey = value_of(B.ym) - sy - value_of(A.ym);
        const double nx = value_of(A.nx) + value_of(B.nx), ny = value_of(A.ny) + value_of(B.ny);
        // (to 1e-4 of the length: enough for meshes read from files with 6-8 digits, while a
        // wrong partner or shift misses by O(1))
        if (!(std::fabs(la - lb) <= 1e-4 * (la + lb) && std::hypot(ex, ey) <= 1e-4 * (la + lb) &&
              std::hypot(nx, ny) <= 1e-4)) {
            *why = "periodic pair " + std::to_string(q) + ": edge b is not edge a moved by the shift";
            return FVLBM_ERR_BAD_BC;
        }
        gap = std::max(gap, std::max(std::fabs(la - lb), std::hypot(ex, ey)) / (0.5 * (la + lb)));
        gap = std::max(gap, std::hypot(nx, ny));
        A.nbr = bside[eb].cell;
        A.back = bside[eb].local;
        A.sx = -sx;
        A.sy = -sy;
        B.nbr = bside[ea].cell;
        B.back = bside[ea].local;
        B.sx = sx;
        B.sy = sy;
        // the glued face is one face: side B takes side A's normal reversed and its length
        B.nx = -A.nx;
        B.ny = -A.ny;
        B.len = A.len;
        glued[ea] = glued[eb] = 1;
    }
    // every face must now be closed
    for (int i = 0; i < nc; ++i) {
        const int nv = m.cell_ptr[i + 1] - m.cell_ptr[i];
        for (int l = 0; l < nv; ++l) {
            const FaceGeo<S> &F = face[4 * static_cast<size_t>(i) + l];
            if (F.nbr == kNone) {
                *why = "cell " + std::to_string(i) + " has an open edge with no boundary record";
                return FVLBM_ERR_BAD_BC;
            }
            if (F.nbr < 0 && bc.bedge_type[-F.nbr - 1] == FVLBM_BC_PERIODIC &&
                !glued[-F.nbr - 1]) {
                *why = "periodic edge without a partner";
                return FVLBM_ERR_BAD_BC;
            }
        }
    }

    // Renumbering: Hilbert order of the centroids (32-bit resolution per axis, so that even
    // wall cells of 1e-6 chord on a 40-chord domain get distinct keys) seeds the block growth
    double x0 = value_of(cx[0]), x1 = x0, y0 = value_of(cy[0]), y1 = y0;
    for (int i = 0; i < nc; ++i) {
        x0 = std::min(x0, value_of(cx[i])); x1 = std::max(x1, value_of(cx[i]));
        y0 = std::min(y0, value_of(cy[i])); y1 = std::max(y1, value_of(cy[i]));
    }
    const double span = std::max(x1 - x0, y1 - y0) + 1e-300;
    const double qmax = 4294967295.0;
    std::vector<std::pair<uint64_t, int>> key(nc);
    for (int i = 0; i < nc; ++i) {
        const uint64_t qx = static_cast<uint64_t>(std::min(qmax, (value_of(cx[i]) - x0) / span * qmax));
        const uint64_t qy = static_cast<uint64_t>(std::min(qmax, (value_of(cy[i]) - y0) / span * qmax));
        key[i] = {hilbert_key(qx, qy), i};
    }
    std::stable_sort(key.begin(), key.end(),
                     [](const auto &a, const auto &b) { return a.first < b.first; });
    // Grow blocks of kBlock cells by breadth-first search over face neighbours, seeded in
    // Hilbert order: each block is a compact patch in the mesh graph (compact in index space
    // even where cells are 1000:1 anisotropic), which keeps the fused kernel's halo rings short.
    {
        std::vector<char> taken(nc, 0);
        std::vector<int> order, queue;
        order.reserve(nc);
        size_t seed = 0;
        while (static_cast<int>(order.size()) < nc) {
            const size_t block_start = order.size();
            const size_t want = std::min<size_t>(kBlock, nc - block_start);
            while (order.size() - block_start < want) {
                while (taken[key[seed].second]) ++seed;
                queue.clear();
                queue.push_back(key[seed].second);
                taken[key[seed].second] = 1;
                size_t head = 0;
                while (head < queue.size() && order.size() - block_start < want) {
                    const int c = queue[head++];
                    order.push_back(c);
                    const int nv = m.cell_ptr[c + 1] - m.cell_ptr[c];
                    for (int l = 0; l < nv; ++l) {
                        const int v = face[4 * static_cast<size_t>(c) + l].nbr;
                        if (v >= 0 && !taken[v]) {
                            taken[v] = 1;
                            queue.push_back(v);
                        }
                    }
                }
                for (size_t q = head; q < queue.size(); ++q) taken[queue[q]] = 0;  // did not fit
            }
        }
        for (int k = 0; k < nc; ++k) key[k].second = order[k];
    }
    PreparedT<S> &P = *out;
    P = PreparedT<S>();
    P.nc = nc;
    P.periodic_gap = gap;
    P.np = (nc + kBlock - 1) / kBlock * kBlock;
    P.n_bedges_in = nbe;
    const size_t np = P.np;
    P.perm.resize(nc);
    std::vector<int> inv(nc);
    for (int k = 0; k < nc; ++k) {
        P.perm[k] = key[k].second;
        inv[key[k].second] = k;
    }
    // boundary faces (non-periodic edges), numbered in input order
    std::vector<int> bface_of_edge(nbe, -1);
    for (int b = 0; b < nbe; ++b) {
        if (glued[b]) continue;
        bface_of_edge[b] = P.nb++;
        P.bedge_of.push_back(b);
    }
    P.bowner.resize(P.nb);
    P.btype.resize(P.nb);
    P.bval.resize(5 * static_cast<size_t>(P.nb));
    P.bnrm.resize(2 * static_cast<size_t>(P.nb));
    P.blen.resize(P.nb);
    for (int f = 0; f < P.nb; ++f) {
        const int b = P.bedge_of[f];
        const FaceGeo<S> &F = face[4 * static_cast<size_t>(bside[b].cell) + bside[b].local];
        P.bowner[f] = inv[bside[b].cell];
        P.btype[f] = bc.bedge_type[b];
        for (int c = 0; c < 5; ++c) P.bval[5 * f + c] = bc.bedge_val[5 * b + c];
        P.bnrm[2 * f] = F.nx;
        P.bnrm[2 * f + 1] = F.ny;
        P.blen[f] = F.len;
    }

    P.nbr.assign(4 * np, kNone);
    P.back.assign(4 * np, -1);
    P.glued.assign(4 * np, 0);
    P.nface.assign(np, 0);
    P.gq.assign(8 * np, S(0.0));
    P.sn.assign(8 * np, S(0.0));
    P.lsq.assign(8 * np, S(0.0));
    P.dvec.assign(8 * np, S(0.0));
    P.rown.assign(8 * np, S(0.0));
    P.rnbr.assign(8 * np, S(0.0));
    P.dinv.assign(4 * np, S(0.0));
    P.area.assign(np, S(0.0));
    P.wdist.assign(np, S(1e30));
    for (int k = 0; k < nc; ++k) {
        const int i = P.perm[k];
        const int nv = m.cell_ptr[i + 1] - m.cell_ptr[i];
        P.area[k] = area[i];
        P.nface[k] = nv;
        for (int l = 0; l < nv; ++l) {  // node positions relative to the centroid
            const int a = m.cell_nodes[m.cell_ptr[i] + l];
            P.gq[(2 * l) * np + k] = xy[2 * a] - cx[i];
            P.gq[(2 * l + 1) * np + k] = xy[2 * a + 1] - cy[i];
        }
        S dx[4], dy[4];
        S mxx = 0, mxy = 0, myy = 0;
        for (int l = 0; l < nv; ++l) {
            const FaceGeo<S> &F = face[4 * static_cast<size_t>(i) + l];
            if (F.nbr >= 0) {
                const S xj = cx[F.nbr] + F.sx, yj = cy[F.nbr] + F.sy;
                P.nbr[l * np + k] = inv[F.nbr];
                P.back[l * np + k] = F.back;
                P.glued[l * np + k] = (F.sx != 0.0 || F.sy != 0.0) ? 1 : 0;
                dx[l] = xj - cx[i];
                dy[l] = yj - cy[i];
                P.rnbr[(2 * l) * np + k] = F.xm - xj;
                P.rnbr[(2 * l + 1) * np + k] = F.ym - yj;
            } else {
                P.nbr[l * np + k] = -(bface_of_edge[-F.nbr - 1] + 1);
                dx[l] = F.xm - cx[i];
                dy[l] = F.ym - cy[i];
            }
            P.sn[(2 * l) * np + k] = F.nx * F.len / area[i];
            P.sn[(2 * l + 1) * np + k] = F.ny * F.len / area[i];
            P.rown[(2 * l) * np + k] = F.xm - cx[i];
            P.rown[(2 * l + 1) * np + k] = F.ym - cy[i];
            P.dinv[l * np + k] = S(1.0) / sqrt(dx[l] * dx[l] + dy[l] * dy[l]);
            mxx += dx[l] * dx[l];
            mxy += dx[l] * dy[l];
            myy += dy[l] * dy[l];
        }
        const S det = mxx * myy - mxy * mxy;
        if (!(det > S(0.0))) {
            *why = "degenerate least-squares stencil at cell " + std::to_string(i);
            return FVLBM_ERR_BAD_MESH;
        }
        for (int l = 0; l < nv; ++l) {
            P.dvec[(2 * l) * np + k] = dx[l];
            P.dvec[(2 * l + 1) * np + k] = dy[l];
            P.lsq[(2 * l) * np + k] = (myy * dx[l] - mxy * dy[l]) / det;
            P.lsq[(2 * l + 1) * np + k] = (mxx * dy[l] - mxy * dx[l]) / det;
        }
    }
    // wall distance: centroid to nearest wall face (brute force over wall faces)
    std::vector<int> walls;
    for (int b = 0; b < nbe; ++b)
        if (!glued[b] && bc.bedge_type[b] == FVLBM_BC_WALL) walls.push_back(b);
    if (!walls.empty()) {
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nc; ++k) {
            const int i = P.perm[k];
            S best = 1e300;
            for (int b : walls) {
                const int a0 = bc.bedge_nodes[2 * b], a1 = bc.bedge_nodes[2 * b + 1];
                best = smin(best, point_segment(cx[i], cy[i], xy[2 * a0], xy[2 * a0 + 1],
                                                xy[2 * a1], xy[2 * a1 + 1]));
            }
            P.wdist[k] = best;
        }
    }
    // time step: dt, or cfl over the largest upwind outflow rate max_i max_alpha
    // sum_m max(e_alpha . n_m, 0) Delta l_m / A_i (forward-Euler limit of first-order upwind).
    // Local time stepping keeps each cell's own cfl / rate_i (steady-state acceleration).
    P.dt = p.dt;
    if (P.dt <= 0.0 || p.local_dt) {
        static const int ex[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        static const int ey[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        std::vector<double> rate_in(nc, 0.0);  // per input cell
        double rate = 0.0;
        for (int i = 0; i < nc; ++i) {
            const int nv = m.cell_ptr[i + 1] - m.cell_ptr[i];
            for (int a = 1; a < kQ; ++a) {
                double s = 0.0;
                for (int l = 0; l < nv; ++l) {
                    const FaceGeo<S> &F = face[4 * static_cast<size_t>(i) + l];
                    const double en = ex[a] * value_of(F.nx) + ey[a] * value_of(F.ny);
                    if (en > 0.0) s += en * value_of(F.len);
                }
                rate_in[i] = std::max(rate_in[i], s / value_of(area[i]));
            }
            rate = std::max(rate, rate_in[i]);
        }
        P.dt = p.cfl / rate;
        if (p.local_dt) {
            P.dt_cell.assign(np, P.dt);  // padding cells: any positive step
            for (int k = 0; k < nc; ++k) P.dt_cell[k] = p.cfl / rate_in[P.perm[k]];
        }
    }
    // initial fields in internal order (padding cells at rest with rho0)
    P.rho_i.assign(np, p.rho0);
    P.u_i.assign(np, 0.0);
    P.v_i.assign(np, 0.0);
    P.k_i.assign(np, 0.0);
    P.w_i.assign(np, 1.0);
    for (int k = 0; k < nc; ++k) {
        const int i = P.perm[k];
        if (p.rho_init) P.rho_i[k] = p.rho_init[i];
        if (p.u_init) P.u_i[k] = p.u_init[i];
        if (p.v_init) P.v_i[k] = p.v_init[i];
        if (p.k_init) P.k_i[k] = p.k_init[i];
        if (p.omega_init) P.w_i[k] = p.omega_init[i];
    }
    return check_prepared(P, why);
}

namespace {

// Area and centroid of cell i as prepare_instance_t forms them (relative to node 0).
template <class S>
void cell_area_centroid(const fvlbm_mesh &m, int i, const S *xy, S *area, S *cx, S *cy) {
    const int p0 = m.cell_ptr[i], nv = m.cell_ptr[i + 1] - p0;
    const int n0 = m.cell_nodes[p0];
    const S ox = xy[2 * n0], oy = xy[2 * n0 + 1];
    S a2 = 0, mx = 0, my = 0;
    for (int l = 0; l < nv; ++l) {
        const int a = m.cell_nodes[p0 + l], b = m.cell_nodes[p0 + (l + 1) % nv];
        const S x0 = xy[2 * a] - ox, y0 = xy[2 * a + 1] - oy;
        const S x1 = xy[2 * b] - ox, y1 = xy[2 * b + 1] - oy;
        const S c = x0 * y1 - x1 * y0;
        a2 += c;
        mx += (x0 + x1) * c;
        my += (y0 + y1) * c;
    }
    *area = S(0.5) * a2;
    *cx = ox + mx / (S(3.0) * a2);
    *cy = oy + my / (S(3.0) * a2);
}

// The geometry of cell i's faces (slot outputs of prepare_instance_t) from its node positions
// xy and its face neighbours' centroids (nbx, nby; slots with nbr[l] < 0 are boundary faces).
template <class S>
struct CellGeo {
    S sn[8], lsq[8], rown[8], rnbr[8], nrm[8], len[4], dinv[4], area;
};

template <class S>
void cell_geometry(const fvlbm_mesh &m, int i, const S *xy, const int *nbr, const S *nbx, const S *nby,
                   CellGeo<S> *G) {
    const int p0 = m.cell_ptr[i], nv = m.cell_ptr[i + 1] - p0;
    S area, cx, cy;
    cell_area_centroid(m, i, xy, &area, &cx, &cy);
    G->area = area;
    S dx[4], dy[4];
    S mxx = 0, mxy = 0, myy = 0;
    for (int l = 0; l < nv; ++l) {
        const int a = m.cell_nodes[p0 + l], b = m.cell_nodes[p0 + (l + 1) % nv];
        const S ex = xy[2 * b] - xy[2 * a], ey = xy[2 * b + 1] - xy[2 * a + 1];
        const S len = sqrt(ex * ex + ey * ey);
        const S nx = ey / len, ny = -ex / len;
        const S xm = S(0.5) * (xy[2 * a] + xy[2 * b]), ym = S(0.5) * (xy[2 * a + 1] + xy[2 * b + 1]);
        if (nbr[l] >= 0) {
            dx[l] = nbx[l] - cx;
            dy[l] = nby[l] - cy;
            G->rnbr[2 * l] = xm - nbx[l];
            G->rnbr[2 * l + 1] = ym - nby[l];
        } else {
            dx[l] = xm - cx;
            dy[l] = ym - cy;
            G->rnbr[2 * l] = G->rnbr[2 * l + 1] = S(0.0);
        }
        G->sn[2 * l] = nx * len / area;
        G->sn[2 * l + 1] = ny * len / area;
        G->rown[2 * l] = xm - cx;
        G->rown[2 * l + 1] = ym - cy;
        G->nrm[2 * l] = nx;
        G->nrm[2 * l + 1] = ny;
        G->len[l] = len;
        G->dinv[l] = S(1.0) / sqrt(dx[l] * dx[l] + dy[l] * dy[l]);
        mxx += dx[l] * dx[l];
        mxy += dx[l] * dy[l];
        myy += dy[l] * dy[l];
    }
    const S det = mxx * myy - mxy * mxy;
    for (int l = 0; l < nv; ++l) {
        G->lsq[2 * l] = (myy * dx[l] - mxy * dy[l]) / det;
        G->lsq[2 * l + 1] = (mxx * dy[l] - mxy * dx[l]) / det;
    }
}

}  // namespace

int geometry_adjoint(const fvlbm_mesh &m, const fvlbm_bc &bc, const GeometryAdjoint &A, double *dxy,
                     std::string *why) {
    const int nc = m.n_cells, nn = m.n_nodes;
    if (bc.n_periodic > 0) {
        *why = "shape adjoint of periodic meshes";
        return FVLBM_ERR_NOT_SUPPORTED;
    }
    // face neighbours (input ids) and boundary edges of every face slot
    std::vector<int> nbr(4 * static_cast<size_t>(nc), kNone);
    std::unordered_map<uint64_t, Side> open;
    open.reserve(static_cast<size_t>(nc) * 3);
    for (int i = 0; i < nc; ++i) {
        const int p0 = m.cell_ptr[i], nv = m.cell_ptr[i + 1] - p0;
        for (int l = 0; l < nv; ++l) {
            const uint64_t id = edge_id(m.cell_nodes[p0 + l], m.cell_nodes[p0 + (l + 1) % nv]);
            auto it = open.find(id);
            if (it == open.end()) {
                open.emplace(id, Side{i, l});
            } else {
                nbr[4 * static_cast<size_t>(i) + l] = it->second.cell;
                nbr[4 * static_cast<size_t>(it->second.cell) + it->second.local] = i;
            }
        }
    }
    for (int b = 0; b < bc.n_bedges; ++b) {
        auto it = open.find(edge_id(bc.bedge_nodes[2 * b], bc.bedge_nodes[2 * b + 1]));
        if (it == open.end()) {
            *why = "boundary edge not on the mesh";
            return FVLBM_ERR_BAD_BC;
        }
        nbr[4 * static_cast<size_t>(it->second.cell) + it->second.local] = -(b + 1);
    }
    std::vector<double> cxv(nc), cyv(nc), dc(2 * static_cast<size_t>(nc), 0.0);
    for (int i = 0; i < nc; ++i) {
        double ar;
        cell_area_centroid(m, i, m.xy, &ar, &cxv[i], &cyv[i]);
    }
    std::fill(dxy, dxy + 2 * static_cast<size_t>(nn), 0.0);
    std::vector<Dual> xyd(2 * static_cast<size_t>(nn));
    for (size_t k = 0; k < xyd.size(); ++k) xyd[k] = Dual(m.xy[k], 0.0);
    for (int i = 0; i < nc; ++i) {
        const int p0 = m.cell_ptr[i], nv = m.cell_ptr[i + 1] - p0;
        const int *nb = nbr.data() + 4 * static_cast<size_t>(i);
        Dual nbx[4], nby[4];
        for (int l = 0; l < nv; ++l)
            if (nb[l] >= 0) {
                nbx[l] = Dual(cxv[nb[l]]);
                nby[l] = Dual(cyv[nb[l]]);
            }
        // adjoint . d(outputs) for the current seed
        auto contract = [&](const CellGeo<Dual> &G) {
            double s = A.area.empty() ? 0.0 : A.area[i] * G.area.d;
            for (int l = 0; l < nv; ++l) {
                const size_t o = (4 * static_cast<size_t>(i) + l) * 2;
                for (int c = 0; c < 2; ++c) {
                    s += A.sn[o + c] * G.sn[2 * l + c].d + A.lsq[o + c] * G.lsq[2 * l + c].d +
                         A.rown[o + c] * G.rown[2 * l + c].d + A.rnbr[o + c] * G.rnbr[2 * l + c].d;
                }
                if (!A.dinv.empty()) s += A.dinv[4 * static_cast<size_t>(i) + l] * G.dinv[l].d;
                if (nb[l] < 0 && nb[l] != kNone) {
                    const int b = -nb[l] - 1;
                    s += A.bnrm[2 * b] * G.nrm[2 * l].d + A.bnrm[2 * b + 1] * G.nrm[2 * l + 1].d +
                         A.blen[b] * G.len[l].d;
                }
            }
            return s;
        };
        CellGeo<Dual> G;
        for (int l = 0; l < nv; ++l) {  // own node coordinates
            const int a = m.cell_nodes[p0 + l];
            for (int c = 0; c < 2; ++c) {
                xyd[2 * a + c].d = 1.0;
                cell_geometry<Dual>(m, i, xyd.data(), nb, nbx, nby, &G);
                xyd[2 * a + c].d = 0.0;
                dxy[2 * a + c] += contract(G);
            }
        }
        for (int l = 0; l < nv; ++l) {  // neighbour centroids
            if (nb[l] < 0) continue;
            for (int c = 0; c < 2; ++c) {
                (c == 0 ? nbx[l] : nby[l]).d = 1.0;
                cell_geometry<Dual>(m, i, xyd.data(), nb, nbx, nby, &G);
                (c == 0 ? nbx[l] : nby[l]).d = 0.0;
                dc[2 * static_cast<size_t>(nb[l]) + c] += contract(G);
            }
        }
    }
    // wall distance: the nearest wall face (first of equals, in input order, as the forward
    // search keeps it) and the point-segment distance's local Jacobian
    if (!A.wdist.empty()) {
        std::vector<int> walls;
        for (int b = 0; b < bc.n_bedges; ++b)
            if (bc.bedge_type[b] == FVLBM_BC_WALL) walls.push_back(b);
        std::vector<int> nearest(walls.empty() ? 0 : nc, -1);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < static_cast<int>(nearest.size()); ++i) {
            if (A.wdist[i] == 0.0) continue;
            double best = 1e300;
            for (int b : walls) {
                const int a0 = bc.bedge_nodes[2 * b], a1 = bc.bedge_nodes[2 * b + 1];
                const double d = point_segment(cxv[i], cyv[i], m.xy[2 * a0], m.xy[2 * a0 + 1], m.xy[2 * a1],
                                               m.xy[2 * a1 + 1]);
                if (d < best) {
                    best = d;
                    nearest[i] = b;
                }
            }
        }
        for (int i = 0; i < static_cast<int>(nearest.size()); ++i) {
            const double lw = A.wdist[i];
            if (lw == 0.0 || nearest[i] < 0) continue;
            const int bw = nearest[i];
            const int a0 = bc.bedge_nodes[2 * bw], a1 = bc.bedge_nodes[2 * bw + 1];
            for (int k = 0; k < 6; ++k) {
                Dual in[6] = {Dual(cxv[i]), Dual(cyv[i]), Dual(m.xy[2 * a0]), Dual(m.xy[2 * a0 + 1]),
                              Dual(m.xy[2 * a1]), Dual(m.xy[2 * a1 + 1])};
                in[k].d = 1.0;
                const double g = lw * point_segment(in[0], in[1], in[2], in[3], in[4], in[5]).d;
                if (k < 2)
                    dc[2 * static_cast<size_t>(i) + k] += g;
                else
                    dxy[2 * (k < 4 ? a0 : a1) + (k & 1)] += g;
            }
        }
    }
    // centroid adjoints to the nodes of their cells
    for (int j = 0; j < nc; ++j) {
        const int p0 = m.cell_ptr[j], nv = m.cell_ptr[j + 1] - p0;
        for (int l = 0; l < nv; ++l) {
            const int a = m.cell_nodes[p0 + l];
            for (int c = 0; c < 2; ++c) {
                xyd[2 * a + c].d = 1.0;
                Dual ar, cx, cy;
                cell_area_centroid<Dual>(m, j, xyd.data(), &ar, &cx, &cy);
                xyd[2 * a + c].d = 0.0;
                dxy[2 * a + c] += dc[2 * static_cast<size_t>(j)] * cx.d + dc[2 * static_cast<size_t>(j) + 1] * cy.d;
            }
        }
    }
    return FVLBM_OK;
}

namespace {

// C(c + r, c), saturated at 2e9
int binom_cr(int c, int r)
{
    double b = 1.0;
    for (int i = 1; i <= c; ++i) b = b * (r + i) / i;
    return b > 2e9 ? 2000000000 : static_cast<int>(b + 0.5);
}

// units u0 .. u0+n-1, the state at u0 in snapshot `from`, snapshots free from index `free`
bool revolve_rec(int u0, int n, int from, int free, int snaps, std::vector<RevolveAction> *out)
{
    if (n <= 0) return true;
    if (n == 1) {
        out->push_back({RevolveAction::kReverse, u0, u0 + 1, from, -1});
        return true;
    }
    const int c = snaps - free;
    if (c <= 0) return false;
    int r = 1;
    while (binom_cr(c, r) < n) ++r;
    const int tail = std::min(n - 1, binom_cr(c - 1, r));
    const int head = n - tail;
    out->push_back({RevolveAction::kAdvance, u0, u0 + head, from, free});
    return revolve_rec(u0 + head, tail, free, free + 1, snaps, out) && revolve_rec(u0, head, from, free, snaps, out);
}

}  // namespace

bool revolve_schedule(int units, int snaps, std::vector<RevolveAction> *out)
{
    out->clear();
    return revolve_rec(0, units, -1, 0, snaps, out);
}

template <class S>
int check_prepared(const PreparedT<S> &P, std::string *why) {
    auto fail = [why](int code, const std::string &msg) {
        *why = "preprocessing check: " + msg;
        return code;
    };
    auto at = [](int k, int m) { return "cell " + std::to_string(k) + " face " + std::to_string(m); };
    const int nc = P.nc, nb = P.nb;
    const size_t np = static_cast<size_t>(P.np), unb = static_cast<size_t>(nb);
    if (nc <= 0 || P.np < nc || P.np % kBlock != 0 || P.np - nc >= kBlock || nb < 0)
        return fail(FVLBM_ERR_BAD_MESH, "cell or face counts");
    const size_t n4 = 4 * np, n8 = 8 * np;
    if (P.perm.size() != static_cast<size_t>(nc) || P.nbr.size() != n4 || P.back.size() != n4 || P.glued.size() != n4 ||
        P.nface.size() != np || P.gq.size() != n8 || P.sn.size() != n8 || P.lsq.size() != n8 ||
        P.dvec.size() != n8 || P.rown.size() != n8 || P.rnbr.size() != n8 || P.dinv.size() != n4 ||
        P.area.size() != np || P.wdist.size() != np || P.bowner.size() != unb ||
        P.btype.size() != unb || P.bval.size() != 5 * unb || P.bnrm.size() != 2 * unb ||
        P.blen.size() != unb || P.bedge_of.size() != unb ||
        !(P.dt_cell.empty() || P.dt_cell.size() == np) || P.rho_i.size() != np ||
        P.u_i.size() != np || P.v_i.size() != np || P.k_i.size() != np || P.w_i.size() != np)
        return fail(FVLBM_ERR_BAD_MESH, "array sizes");
    std::vector<char> seen(nc, 0);
    for (int k = 0; k < nc; ++k) {
        const int i = P.perm[k];
        if (i < 0 || i >= nc || seen[i]) return fail(FVLBM_ERR_BAD_MESH, "cell order is not a permutation");
        seen[i] = 1;
    }
    for (int f = 0; f < nb; ++f) {
        if (P.bedge_of[f] < 0 || P.bedge_of[f] >= P.n_bedges_in || (f > 0 && P.bedge_of[f] <= P.bedge_of[f - 1]))
            return fail(FVLBM_ERR_BAD_BC, "boundary face " + std::to_string(f) + ": input edge index");
        if (P.btype[f] < FVLBM_BC_WALL || P.btype[f] >= FVLBM_BC_PERIODIC)
            return fail(FVLBM_ERR_BAD_BC, "boundary face " + std::to_string(f) + ": type");
    }
    // Connectivity: every index a kernel gathers through is in range, interior links are mutual
    // (the neighbour's slot `back` points back here), every boundary face is one cell face of its
    // owner, slots past a cell's faces and the padding cells are empty.
    std::vector<long long> bslot(unb, -1);
    for (size_t k = 0; k < np; ++k) {
        const int nf = P.nface[k];
        const double A = value_of(P.area[k]);
        if (k >= static_cast<size_t>(nc)) {
            if (nf != 0 || A != 0.0) return fail(FVLBM_ERR_BAD_MESH, "padding cell " + std::to_string(k) + " is not inert");
        } else if (nf != 3 && nf != 4) {
            return fail(FVLBM_ERR_BAD_MESH, "cell " + std::to_string(k) + ": face count");
        } else if (!(A > 0.0 && std::isfinite(A))) {
            return fail(FVLBM_ERR_BAD_MESH, "cell " + std::to_string(k) + ": area");
        }
        for (int m = 0; m < 4; ++m) {
            const size_t s = static_cast<size_t>(m) * np + k;
            const int v = P.nbr[s], b = P.back[s];
            if (m >= nf) {
                if (v != kNone || b != -1) return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": slot past the faces is not empty");
                continue;
            }
            if (v >= 0) {
                if (v >= nc || b < 0 || b >= P.nface[v] || P.nbr[static_cast<size_t>(b) * np + v] != static_cast<int>(k) ||
                    P.back[static_cast<size_t>(b) * np + v] != m)
                    return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": neighbour link is not mutual");
            } else if (v == kNone) {
                return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": open face");
            } else {
                const int f = -(v + 1);
                if (f >= nb || b != -1 || P.bowner[f] != static_cast<int>(k) || bslot[f] >= 0)
                    return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": boundary face link");
                bslot[f] = static_cast<long long>(s);
            }
        }
    }
    for (int f = 0; f < nb; ++f)
        if (bslot[f] < 0) return fail(FVLBM_ERR_BAD_MESH, "boundary face " + std::to_string(f) + " is no cell face");
    // Geometry: the arrays agree with the node positions (gq) and with each other across every
    // face.  Tolerances are relative (1e-6) and far above rounding on cells down to 1e-6 of the
    // domain; a wrong slot, sign or operand misses them by O(1).
    constexpr double tol = 1e-6;
    // Across a periodic pair the two edges agree only to the gluing tolerance (1e-4), so on
    // glued faces (only there) the checks that compare a face with the neighbour's own copy
    // of it use a looser one.
    constexpr double tol_link = 1e-3;
    auto V = [np](const std::vector<S> &a, int c, size_t k) { return value_of(a[static_cast<size_t>(c) * np + k]); };
    for (int k = 0; k < nc; ++k) {
        const int nf = P.nface[k];
        const double A = value_of(P.area[k]);
        double gx[4], gy[4], h = 0.0;
        for (int m = 0; m < nf; ++m) {
            gx[m] = V(P.gq, 2 * m, k);
            gy[m] = V(P.gq, 2 * m + 1, k);
            if (!(std::isfinite(gx[m]) && std::isfinite(gy[m]))) return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": node position");
            h = std::max(h, std::hypot(gx[m], gy[m]));
        }
        double a2 = 0.0, mx = 0.0, my = 0.0;  // shoelace area and first moment about the centroid
        for (int m = 0; m < nf; ++m) {
            const int m1 = (m + 1) % nf;
            const double c = gx[m] * gy[m1] - gx[m1] * gy[m];
            a2 += c;
            mx += (gx[m] + gx[m1]) * c;
            my += (gy[m] + gy[m1]) * c;
        }
        if (!(std::fabs(0.5 * a2 - A) <= tol * A))
            return fail(FVLBM_ERR_BAD_MESH, "cell " + std::to_string(k) + ": area disagrees with the nodes");
        if (!(std::hypot(mx, my) <= tol * h * 3.0 * a2))
            return fail(FVLBM_ERR_BAD_MESH, "cell " + std::to_string(k) + ": nodes are not relative to the centroid");
        double E[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, T[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
        for (int m = 0; m < nf; ++m) {
            const int m1 = (m + 1) % nf;
            const double tx = gx[m1] - gx[m], ty = gy[m1] - gy[m], L = std::hypot(tx, ty);
            const double nlx = V(P.sn, 2 * m, k) * A, nly = V(P.sn, 2 * m + 1, k) * A;
            const int v = P.nbr[static_cast<size_t>(m) * np + k];
            const bool per = P.glued[static_cast<size_t>(m) * np + k] != 0;
            if (!(std::hypot(nlx - ty, nly + tx) <= (per ? tol_link : tol) * L))
                return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": n dl is not the outward normal of the edge");
            const double rx = V(P.rown, 2 * m, k), ry = V(P.rown, 2 * m + 1, k);
            if (!(std::hypot(rx - 0.5 * (gx[m] + gx[m1]), ry - 0.5 * (gy[m] + gy[m1])) <= tol * h))
                return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": face midpoint");
            const double dx = V(P.dvec, 2 * m, k), dy = V(P.dvec, 2 * m + 1, k), d = std::hypot(dx, dy);
            const double qx = V(P.rnbr, 2 * m, k), qy = V(P.rnbr, 2 * m + 1, k);
            const double di = value_of(P.dinv[static_cast<size_t>(m) * np + k]);
            if (!(d > 0.0 && std::isfinite(d) && std::fabs(di * d - 1.0) <= 1e-12))
                return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": centroid offset or 1/|d|");
            if (v < 0) {  // boundary face: d is the offset to the face midpoint
                if (dx != rx || dy != ry || qx != 0.0 || qy != 0.0)
                    return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": boundary face offsets");
                const int f = -(v + 1);
                const double bl = value_of(P.blen[f]), bx = value_of(P.bnrm[2 * f]), by = value_of(P.bnrm[2 * f + 1]);
                if (!(std::fabs(std::hypot(bx, by) - 1.0) <= 1e-12 && std::hypot(bx * bl - nlx, by * bl - nly) <= tol * L))
                    return fail(FVLBM_ERR_BAD_MESH, "boundary face " + std::to_string(f) + ": normal or length");
            } else {  // interior (or periodic) face, seen again from the neighbour's slot b
                const int b = P.back[static_cast<size_t>(m) * np + k];
                const double Av = value_of(P.area[v]);
                const double vx = V(P.dvec, 2 * b, v), vy = V(P.dvec, 2 * b + 1, v);
                const double ox = V(P.rown, 2 * b, v), oy = V(P.rown, 2 * b + 1, v);
                const double wx = V(P.sn, 2 * b, v) * Av, wy = V(P.sn, 2 * b + 1, v) * Av;
                if (!(std::hypot(dx + vx, dy + vy) <= tol * d))
                    return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": d is not the reverse of the neighbour's");
                if (!(std::hypot(dx - (rx - qx), dy - (ry - qy)) <= tol * (std::hypot(rx, ry) + std::hypot(qx, qy))) ||
                    !(std::hypot(qx - ox, qy - oy) <= (per ? tol_link : tol) * (std::hypot(qx, qy) + std::hypot(ox, oy) + L)))
                    return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": neighbour-side face offset");
                if (!(std::hypot(nlx + wx, nly + wy) <= tol * L))
                    return fail(FVLBM_ERR_BAD_MESH, at(k, m) + ": n dl is not the reverse of the neighbour's");
            }
            const double w[2] = {V(P.lsq, 2 * m, k), V(P.lsq, 2 * m + 1, k)}, dd[2] = {dx, dy};
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 2; ++c) {
                    E[a][c] += w[a] * dd[c];
                    T[a][c] += std::fabs(w[a] * dd[c]);
                }
        }
        // least-squares weights W_m = M^{-1} d_m reproduce linear fields: sum_m W_m d_m^T = I
        for (int a = 0; a < 2; ++a)
            for (int c = 0; c < 2; ++c)
                if (!(std::fabs(E[a][c] - (a == c ? 1.0 : 0.0)) <= tol * std::max(T[a][c], 1.0)))
                    return fail(FVLBM_ERR_BAD_MESH, "cell " + std::to_string(k) + ": least-squares weights");
        const double wd = value_of(P.wdist[k]);
        if (!(wd >= 0.0 && wd <= 1e30)) return fail(FVLBM_ERR_BAD_MESH, "cell " + std::to_string(k) + ": wall distance");
    }
    if (!(P.dt > 0.0 && std::isfinite(P.dt))) return fail(FVLBM_ERR_BAD_PARAM, "time step");
    for (double t : P.dt_cell)
        if (!(t > 0.0 && std::isfinite(t))) return fail(FVLBM_ERR_BAD_PARAM, "local time step");
    return FVLBM_OK;
}

template int prepare_instance_t<double>(const fvlbm_mesh &, const fvlbm_bc &, const fvlbm_params &,
                                        const double *, PreparedT<double> *, std::string *);
template int prepare_instance_t<Dual>(const fvlbm_mesh &, const fvlbm_bc &, const fvlbm_params &,
                                      const Dual *, PreparedT<Dual> *, std::string *);
template int check_prepared<double>(const PreparedT<double> &, std::string *);
template int check_prepared<Dual>(const PreparedT<Dual> &, std::string *);

}  // namespace fvlbm

extern "C" int fvlbm_cell_geometry(const fvlbm_mesh *mesh, const fvlbm_bc *bc,
                                   const fvlbm_params *params, double *area, double *wdist) {
    if (!mesh || !bc || !params) return FVLBM_ERR_BAD_PARAM;
    fvlbm::Prepared P;
    std::string msg;
    const int rc = fvlbm::prepare_instance(*mesh, *bc, *params, &P, &msg);
    if (rc != FVLBM_OK) return rc;
    for (int k = 0; k < P.nc; ++k) {  // internal order -> input order
        const int c = P.perm[k];
        if (area) area[c] = P.area[k];
        if (wdist) wdist[c] = P.wdist[k];
    }
    return FVLBM_OK;
}

extern "C" int fvlbm_check_mesh(const fvlbm_mesh *mesh, const fvlbm_bc *bc, const fvlbm_params *params,
                                double *dt, char *why, int why_len) {
    std::string msg;
    int rc = FVLBM_OK;
    if (!mesh || !bc || !params) {
        rc = FVLBM_ERR_BAD_PARAM;
        msg = "NULL argument";
    } else if (params->precision != FVLBM_FP64 && params->precision != FVLBM_FP32_DEV &&
               params->precision != FVLBM_FP64_TANGENT) {
        rc = FVLBM_ERR_BAD_PARAM;
        msg = "unknown precision";
    } else if (params->scheme != 0 && params->scheme != 1) {
        rc = FVLBM_ERR_BAD_PARAM;
        msg = "unknown scheme";
    } else {
        fvlbm::Prepared P;
        rc = fvlbm::prepare_instance(*mesh, *bc, *params, &P, &msg);
        if (rc == FVLBM_OK && dt) *dt = P.dt;
    }
    if (why && why_len > 0) {
        const size_t n = std::min(msg.size(), static_cast<size_t>(why_len - 1));
        std::memcpy(why, msg.data(), n);
        why[n] = '\0';
    }
    return rc;
}
