// fvlbm_internal.h -- host-side preprocessed mesh shared by the two translation units of the
// library (mesh preprocessing in fvlbm_host.cpp, device code and entry points in
// fvlbm_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "fvlbm.h"
#include "fvlbm_dual.h"

namespace fvlbm {

constexpr int kQ = 9;          // D2Q9
constexpr int kTile = 128;     // cells per thread block of the per-cell kernels
#ifndef FVLBM_FUSED_BLOCK
#define FVLBM_FUSED_BLOCK 256
#endif
constexpr int kBlock = FVLBM_FUSED_BLOCK;  // cells per block of the fused stage kernel (a
                                           // multiple of kTile); instances are padded to a
                                           // multiple of kBlock
static_assert(kBlock % kTile == 0, "fused block must be a whole number of tiles");
constexpr int kNone = INT32_MIN;  // empty face slot (triangles have 3 faces, padding cells 0)

// One instance after preprocessing, in the library's internal cell order (Hilbert order of the
// cell centroids), padded with inert cells (no faces, zero area) to a multiple of kBlock.
// Face slot m of cell i is stored at [m * np + i] (vectors: [(2 m + c) * np + i]) so that one
// thread per cell reads every array with unit stride.  S is the scalar of the geometry: double,
// or Dual when the derivative of the geometry with respect to node positions is wanted.
template <class S>
struct PreparedT {
    int nc = 0;                 // real cells
    int np = 0;                 // padded cells
    int nb = 0;                 // boundary faces (non-periodic boundary edges)
    int n_bedges_in = 0;        // boundary edges in the input (including periodic ones)
    std::vector<int> perm;      // internal id -> input cell id   [nc]
    std::vector<int> nbr;       // [4 np]  neighbour internal id, -(b+1) for boundary face b, kNone
    std::vector<int> back;      // [4 np]  face slot of this face in the neighbour's list (or -1)
    std::vector<int> nface;     // [np]    3 or 4 (0 for padding cells)
    std::vector<S> gq;     // [8 np]  node k position minus centroid (x, y) for k < nface;
                                //         face m joins nodes m and (m + 1) mod nface
    std::vector<S> sn;     // [8 np]  n * Delta l / A of face m, out of the cell
    std::vector<S> lsq;    // [8 np]  least-squares weight W_m = M^{-1} d_m
    std::vector<S> dvec;   // [8 np]  d_m: neighbour centroid (+ shift) or face midpoint,
                                //         minus own centroid
    std::vector<S> rown;   // [8 np]  face midpoint - own centroid
    std::vector<S> rnbr;   // [8 np]  face midpoint - (neighbour centroid + periodic shift)
    std::vector<S> dinv;   // [4 np]  1 / |d_m| (SST central diffusion distance)
    std::vector<unsigned char> glued;  // [4 np] 1 where face m joins a periodic partner
    std::vector<S> area;   // [np]    0 for padding cells
    std::vector<S> wdist;  // [np]    distance to the nearest wall face (1e30 if none)
    // boundary faces, ordered by input boundary-edge index (periodic edges dropped)
    std::vector<int> bowner;    // internal owner cell
    std::vector<int> btype;     // FVLBM_BC_*
    std::vector<double> bval;   // [5 nb] rho_b, u_b, v_b, k_b, omega_b
    std::vector<S> bnrm;   // [2 nb] unit normal out of the fluid
    std::vector<S> blen;   // [nb]
    std::vector<int> bedge_of;  // [nb] input boundary-edge index of each boundary face
    double dt = 0.0;            // the instance's step (local stepping: the smallest dt_i)
    double periodic_gap = 0.0;  // largest mismatch of a glued periodic pair, relative to the
                                // edge length (0 without periodic pairs; ~1e-16 for exact ones)
    std::vector<double> dt_cell;  // [np] local time stepping: dt_i of each cell; empty otherwise
    std::vector<double> rho_i, u_i, v_i, k_i, w_i;  // initial fields, internal order [np]
};

using Prepared = PreparedT<double>;

// Validates and preprocesses one (mesh, bc, params) triple, with node positions xy (the mesh's
// own, or the same positions carrying derivatives).  Returns FVLBM_OK or an error code, with a
// message in *why.  The cell order and the time step depend on the values only.
template <class S>
int prepare_instance_t(const fvlbm_mesh &m, const fvlbm_bc &bc, const fvlbm_params &p, const S *xy,
                       PreparedT<S> *out, std::string *why);
extern template int prepare_instance_t<double>(const fvlbm_mesh &, const fvlbm_bc &,
                                               const fvlbm_params &, const double *,
                                               PreparedT<double> *, std::string *);
extern template int prepare_instance_t<Dual>(const fvlbm_mesh &, const fvlbm_bc &,
                                             const fvlbm_params &, const Dual *, PreparedT<Dual> *,
                                             std::string *);

// Consistency checks on a prepared instance, run at the end of prepare_instance_t: every index
// the kernels gather through is in range (neighbours, back slots, boundary faces, owners), the
// face links are mutual, padding cells are inert, and the geometry arrays agree with the node
// positions and with each other across every face (n dl, midpoints, centroid offsets, 1 / |d|,
// sum_m W_m d_m^T = I).  Returns FVLBM_OK or an error code with a message in *why.
template <class S>
int check_prepared(const PreparedT<S> &P, std::string *why);
extern template int check_prepared<double>(const PreparedT<double> &, std::string *);
extern template int check_prepared<Dual>(const PreparedT<Dual> &, std::string *);

inline int prepare_instance(const fvlbm_mesh &m, const fvlbm_bc &bc, const fvlbm_params &p,
                            Prepared *out, std::string *why) {
    return prepare_instance_t<double>(m, bc, p, m.xy, out, why);
}

// Adjoints of the geometry arrays a step reads, in input order: for face l of input cell i
// (joining its nodes l and l + 1), entry (4 i + l) * 2 + c of sn, lsq, rown, rnbr (c = x, y) and
// entry 4 i + l of dinv; wdist[i] and area[i]; for input boundary edge b, bnrm[2 b + c] and
// blen[b] (periodic edges: unused).  dinv, wdist and area may be empty (only the SST and the
// limiter on grad f read them).
struct GeometryAdjoint {
    std::vector<double> sn, lsq, rown, rnbr, bnrm, blen, dinv, wdist, area;
};

// Reverse mode of the preprocessing above with respect to the node positions: dxy[2 n_nodes] =
// sum over the arrays of adjoint x d(array)/d(x, y), for the areas, centroids, face normals,
// lengths and midpoints, face offsets, least-squares weights, 1 / |d| and the wall distance as
// prepare_instance_t forms them (each cell's local Jacobian by dual numbers, the neighbour
// centroids' adjoints carried to their cells' nodes; the wall distance through its nearest wall
// face).  Meshes with periodic pairs: FVLBM_ERR_NOT_SUPPORTED.
int geometry_adjoint(const fvlbm_mesh &m, const fvlbm_bc &bc, const GeometryAdjoint &A, double *dxy,
                     std::string *why);

// Binomial checkpoint schedule (revolve) for reversing `units` units of forward work with
// `snaps` state snapshots.  Snapshot -1 is the initial state, always available.  Actions, in
// order:
//   kAdvance: run units [u0, u1) from snapshot `from` (holding the state at u0) and store the
//             state at u1 in snapshot `to`;
//   kReverse: run unit u0 from snapshot `from` keeping its stage values, then reverse it.
// Units are reversed last to first.  With c free snapshots and n units the least r with
// C(c + r, c) >= n is taken: the head of the range is advanced to a snapshot, the tail
// (C(c - 1 + r, c - 1) units at most) reversed with c - 1 snapshots, then the head with c.
// Returns false if the units cannot be reversed (no snapshot for a range of two units or more).
struct RevolveAction {
    enum Kind { kAdvance, kReverse } kind;
    int u0, u1, from, to;
};
bool revolve_schedule(int units, int snaps, std::vector<RevolveAction> *out);

}  // namespace fvlbm
