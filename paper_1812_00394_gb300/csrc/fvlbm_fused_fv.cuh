// fvlbm_fused_fv.cuh -- the face-value form of the fused IMEX stage kernel (included by
// fvlbm_kernels.cu after the common device helpers).
//
// What one stage computes is unchanged: least-squares gradients of f^(J) (Step 2), the upwind
// linear face values f_{alpha,bc} = f_up + grad f_up . (x_f - x_up) and the convection term of
// Eq. (advection), then the local stage algebra (Eqs. (sumimeximplicitnew), (fnewstage),
// (imextwo)).  What changes is who forms the face values.
//
// For a face with normal n the nine directions split into the rest direction (no flux) and
// four opposite pairs (alpha, alpha-bar), e_alphabar = -e_alpha, so that e_alphabar . n =
// -e_alpha . n: of every pair exactly one direction leaves the cell through the face (its
// upwind side is the cell itself) and the other enters it (its upwind side is the neighbour).
// Each cell therefore has, per face, four "outgoing" face values -- one per pair -- and the
// neighbour's incoming values at that face are exactly the neighbour's outgoing values at the
// same face.  So every cell of a block (and of its first ring) forms its four outgoing values
// per face once, right after its gradient, and publishes them in shared memory; the flux of a
// cell then reads, per face, its own four values and its neighbour's four (one 16-byte load
// each) instead of gathering the neighbour's f and gradient direction by direction.  Each face
// value is formed once and read by both cells of the face, so the two cells see bit-identical
// values.  Which member of a pair leaves through a face is decided once on the host (FP64
// geometry, e_alpha . n >= 0 on one side of the face and the complement on the other side), so
// the two sides always agree.
//
// Work items: a block of 256 consecutive cells, or -- where its halo would not fit the
// shared-memory budget -- a half or a quarter of one (an instance's cells are padded to a
// multiple of 256, so no item straddles two instances).  One CTA of 256 threads per item.
//
// Layouts for the stages of this form.  f^n stays structure-of-arrays (shared with the rest of
// the library).  The stage values f^(2), f^(3) that stages 1 and 2 write and stages 2 and 3
// read are cell-major: alpha = 1..8 in pair order (1,3)(2,4)(5,7)(6,8) in one 32-byte row per
// cell (its two halves swapped where bit 2 of the cell index is set), then f_0 of every cell,
// so that an item's own rows are one contiguous bulk copy and a halo cell's eight moving
// directions are one 32-byte sector.  The geometry the kernel reads
// (node offsets q[8] and least-squares weights W[8]) is likewise one 64-byte row per cell.
//
// Staging, all issued before any wait: the item's own rows (its stage values, its accumulator
// rows and tau) by bulk copies on one mbarrier, shared out over the warps; the halo rows, the
// adjacency, the ring-1 geometry and the instance parameters by cp.async; the item cell's own
// geometry straight into registers.  A CTA's first loads (its halo ids and its header) do not
// depend on each other, so the gathers wait on two memory round trips.  Stage 1 takes
// its own f^n rows from the accumulator copy (the algebra reads them there too) and relaxes
// every staged cell to f^(1) on chip (Eq. (fnewstage), J = 1), so no f^(1) array passes
// through HBM and f^n is never recovered from a rounded f^(1).
//
// FP32 arithmetic runs on packed pairs (fma.rn.f32x2): the two members of a pair share every
// geometric factor, so the gradient and face-value updates are one packed FMA per pair.

// Shared-memory capacity of the face-value kernel (cells): ring-1 + ring-2 + item cells,
// item + ring-1 cells.  256-cell blocks whose halo exceeds it are split.
constexpr int kFvThreads = 256;
constexpr int kFvEcap = 448;
constexpr int kFvGcap = 352;

// Adjacency word of the face-value kernel (cell-major: 4 words per cell):
//   0xFFFFFFFF: no face; bit 31 set: boundary face (low 31 bits: global boundary face index);
//   else: local index (bits 0-15) | back slot (16-17) | outgoing bits (18-21), bit 18 + p set
//   when the first member of pair p leaves this cell through the face.
constexpr unsigned kFvNone = 0xFFFFFFFFu;
constexpr unsigned kFvBnd = 0x80000000u;

// Halo slots of an item in the fixed-stride table: a 256-cell item has at most
// kFvEcap - 256 halo cells; the larger halos of split items continue in an overflow table.
constexpr int kFvHs = kFvEcap - kFvThreads;

// The item tables are laid out so that a CTA can issue its first loads -- the item's halo ids
// and its header -- together, from its item index alone: the halo ids and the adjacency sit at
// fixed strides per item, and the header carries what the later steps need.  Staging then
// waits on two memory round trips (ids, then the rows they name) instead of three.
struct FvItems {
    const int4 *__restrict__ hdr;       // [nitem]: base cell, cells | ring-1 cells << 16,
                                        // instance, overflow offset (-1: none)
    const int *__restrict__ halo;       // [nitem][kFvHs] global ids, ring 1 then ring 2, -1 after
    const int *__restrict__ ovf;        // halo slots kFvHs.. of the items that have them
    const uint4 *__restrict__ adj;      // [nitem][kFvGcap] adjacency of item and ring-1 cells
    int *__restrict__ err;              // set to 1 if the bulk-copy wait gave up
    long long wait_first;               // polls of that wait (fvlbm_set_wait_limit)
    int item0;                          // first item of this launch (CTA b takes item0 + b)
};

// Pair p: first members alpha = 1, 2, 5, 6 and their opposites 3, 4, 7, 8.
__host__ __device__ constexpr int fv_first(int p) { return p == 0 ? 1 : (p == 1 ? 2 : (p == 2 ? 5 : 6)); }
__host__ __device__ constexpr int fv_second(int p) { return p == 0 ? 3 : (p == 1 ? 4 : (p == 2 ? 7 : 8)); }
// Position of alpha (1..8) in a pair-ordered row of 8: (1,3)(2,4)(5,7)(6,8).
__host__ __device__ constexpr int fv_pos(int a) {
    return a == 1 ? 0 : (a == 3 ? 1 : (a == 2 ? 2 : (a == 4 ? 3 : (a == 5 ? 4 : (a == 7 ? 5 : (a == 6 ? 6 : 7))))));
}

// e_first(p) . (x, y)
template <class T>
__device__ __forceinline__ T fv_en(int p, T x, T y) {
    return p == 0 ? x : (p == 1 ? y : (p == 2 ? x + y : y - x));
}

// A pair of values (first member, opposite member) with packed FP32 arithmetic where available.
template <class T>
struct FvPair;
template <>
struct FvPair<float> {
    using V = float2;
    static __device__ __forceinline__ V make(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ V bcast(float a) { return make_float2(a, a); }
};
template <>
struct FvPair<double> {
    using V = double2;
    static __device__ __forceinline__ V make(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) {
        return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
    }
    static __device__ __forceinline__ V bcast(double a) { return make_double2(a, a); }
};

// Shared-memory layout (bytes):
//   sf  [kFvEcap][8]   staged f (moving directions, pair order, halves swapped on bit 2 of
//                      the row), one row per item / ring cell
//   sf0 [kFvEcap]      staged f_0
//   st  [2][kFvEcap]   stage 1: tau and the time step of every staged halo cell
//   sv  [kFvGcap][16]  outgoing face values, 4 per face slot; 16-byte chunk m of row c sits at
//                      chunk m ^ ((c >> 1) & 3).  Before the face values are written, the
//                      rows of ring-1 cells hold their geometry in the same swizzled chunks
//                      (q[0..3], q[4..7], W[0..3], W[4..7])
//   sa  [kFvGcap]      adjacency words (uint4)
//   sacc [19][256]     the item's rows for the stage algebra, structure of arrays: stage 1
//                      f^n; stage 2 B and C; stage 3 C; then tau
//   the item's instance parameters (copied during staging, read by the stage algebra)
//   one mbarrier for the bulk copies
template <class T>
struct FvSmem {
    static constexpr size_t sf = 0;
    static constexpr size_t sf0 = sf + size_t(kFvEcap) * 8 * sizeof(T);
    static constexpr size_t st = sf0 + ((size_t(kFvEcap) * sizeof(T) + 15) / 16) * 16;
    static constexpr size_t sv = st + 2 * size_t(kFvEcap) * sizeof(T);
    static constexpr size_t sa = sv + size_t(kFvGcap) * 16 * sizeof(T);
    static constexpr size_t sacc = sa + size_t(kFvGcap) * 16;
    static constexpr size_t ip = sacc + size_t(2 * kQ + 1) * kFvThreads * sizeof(T);
    static constexpr size_t bar = ip + sizeof(InstParam);
    static constexpr size_t bytes = bar + 16;
};

// element offset of face slot m in row c of sv
__device__ __forceinline__ int fv_sv_off(int c, int m) { return c * 16 + 4 * (m ^ ((c >> 1) & 3)); }

// Rows of 8 (staged in shared memory, and the cell-major stage values in global memory) keep
// their two 4-value halves swapped when bit 2 of the row index is set: consecutive rows then
// spread over all banks, and since items start at multiples of 64 cells the item rows keep
// the same bit in both places (one bulk copy moves them unchanged).
__host__ __device__ __forceinline__ int fv_half(int j, int h) { return h ^ ((j >> 2) & 1); }

// Load the 8 moving directions of staged row j as 4 pairs.
template <class T>
__device__ __forceinline__ void fv_load_row(const T *sf, int j, typename FvPair<T>::V *o) {
    using PV = FvPair<T>;
    const T *lo_p = sf + j * 8 + 4 * fv_half(j, 0);
    const T *hi_p = sf + j * 8 + 4 * fv_half(j, 1);
    if constexpr (sizeof(T) == 4) {
        const float4 lo = *reinterpret_cast<const float4 *>(lo_p);
        const float4 hi = *reinterpret_cast<const float4 *>(hi_p);
        o[0] = PV::make(lo.x, lo.y);
        o[1] = PV::make(lo.z, lo.w);
        o[2] = PV::make(hi.x, hi.y);
        o[3] = PV::make(hi.z, hi.w);
    } else {
        o[0] = *reinterpret_cast<const double2 *>(lo_p);
        o[1] = *reinterpret_cast<const double2 *>(lo_p + 2);
        o[2] = *reinterpret_cast<const double2 *>(hi_p);
        o[3] = *reinterpret_cast<const double2 *>(hi_p + 2);
    }
}
// element offset of pair p in row j
__device__ __forceinline__ int fv_pair_off(int j, int p) { return j * 8 + 4 * fv_half(j, p >> 1) + 2 * (p & 1); }
// element offset of alpha (1..8) in row j
__device__ __forceinline__ int fv_alpha_off(int j, int a) {
    const int pos = fv_pos(a);
    return j * 8 + 4 * fv_half(j, pos >> 2) + (pos & 3);
}

// 16-byte vector load of geometry (rows of 16 values, 16-byte aligned) into v[0..7], w[0..7]
template <class T>
__device__ __forceinline__ void fv_load_geo_row(const T *__restrict__ g, T *q, T *w) {
    if constexpr (sizeof(T) == 4) {
        const float4 *g4 = reinterpret_cast<const float4 *>(g);
        const float4 a = g4[0], b = g4[1], c = g4[2], d = g4[3];
        q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
        q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w;
        w[0] = c.x; w[1] = c.y; w[2] = c.z; w[3] = c.w;
        w[4] = d.x; w[5] = d.y; w[6] = d.z; w[7] = d.w;
    } else {
        const double2 *g2 = reinterpret_cast<const double2 *>(g);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double2 x = g2[k], y = g2[4 + k];
            q[2 * k] = x.x; q[2 * k + 1] = x.y;
            w[2 * k] = y.x; w[2 * k + 1] = y.y;
        }
    }
}

template <class T>
__device__ __forceinline__ void fv_load_vals(const T *sv, int c, int m, T *v) {
    const T *p = sv + fv_sv_off(c, m);
    if constexpr (sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
        const double2 a = *reinterpret_cast<const double2 *>(p);
        const double2 b = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

template <class T>
__device__ __forceinline__ void fv_store_vals(T *sv, int c, int m, const T *v) {
    T *p = sv + fv_sv_off(c, m);
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
    }
}

// Boundary face values (boundary_values) on boundary face bf of a cell whose f is given as 4
// pairs and f_0, as 4 pairs.  The face's type and (rho, u, v) are read kept in L2, like the
// item tables: a few hundred kB read once per launch by the items along the boundaries.
template <class T>
__device__ __forceinline__ void fv_boundary_pairs(const Geo<T> &G, int bf, T nx, T ny,
                                                  const typename FvPair<T>::V *fc, T f0, T rho0,
                                                  typename FvPair<T>::V *out) {
    using PV = FvPair<T>;
    const unsigned long long keep = l2_keep_policy();
    const int type = ld_keep(G.btype + bf, keep);
    T bval[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) bval[c] = ld_keep(G.bval + static_cast<size_t>(c) * G.nbt + bf, keep);
    const int nbt = 1;
    T fcs[kQ], fb[kQ], dr, r, u, v;
    fcs[0] = f0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        fcs[fv_first(p)] = fc[p].x;
        fcs[fv_second(p)] = fc[p].y;
    }
    moments(fcs, rho0, dr, r, u, v);
    boundary_values(type, bval, 0, nbt, nx, ny, fcs, dr, r, u, v, rho0, fb);
#pragma unroll
    for (int p = 0; p < 4; ++p) out[p] = PV::make(fb[fv_first(p)], fb[fv_second(p)]);
}

// Stage 1: f^(1) = [f^n + (dt/tau)/4 f^eq(f^n)] / (1 + (dt/tau)/4) (Eq. (fnewstage), J = 1)
// of a cell given as f[9] (alpha order), written to staged row e.
template <class T>
__device__ __forceinline__ void fv_relax_to_row(T *f, T *sf, T *sf0, int e, T rho0, T dt, T tau_e,
                                                T *eq_out = nullptr) {
    relax9(f, rho0, dt, tau_e, eq_out);
    sf0[e] = f[0];
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(sf + e * 8 + 4 * fv_half(e, 0)) = make_float4(f[1], f[3], f[2], f[4]);
        *reinterpret_cast<float4 *>(sf + e * 8 + 4 * fv_half(e, 1)) = make_float4(f[5], f[7], f[6], f[8]);
    } else {
#pragma unroll
        for (int a = 1; a < kQ; ++a) sf[fv_alpha_off(e, a)] = f[a];
    }
}

// End node of face m of a cell (m compile-time): node m + 1, wrapping to node 0 after the last
// face; selects between static indices keep q in registers.
#define FV_END_X(m) ((m) == 3 ? q[0] : ((m) == 2 && tri ? q[0] : q[2 * (m) + 2]))
#define FV_END_Y(m) ((m) == 3 ? q[1] : ((m) == 2 && tri ? q[1] : q[2 * (m) + 3]))

// Gradient (Step 2) and outgoing face values of item cell c.  q: node positions relative to
// the centroid; lw: least-squares weights W_m = M^{-1} d_m (x, y per face slot); w: adjacency.
template <class T>
__device__ __forceinline__ void fv_cell(int c, const T *q, const T *lw, const uint4 &w4,
                                        const T *__restrict__ sf, T f0, T *__restrict__ sv,
                                        const Geo<T> &G, T rho0) {
    using PV = FvPair<T>;
    using V = typename PV::V;
    const unsigned w[4] = {w4.x, w4.y, w4.z, w4.w};
    V fc[4];
    fv_load_row(sf, c, fc);
    const bool tri = w[3] == kFvNone;
    V gx[4], gy[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) gx[p] = gy[p] = PV::bcast(T(0));
    const V mone = PV::bcast(T(-1));
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (w[m] == kFvNone) continue;
        const V wx = PV::bcast(lw[2 * m]), wy = PV::bcast(lw[2 * m + 1]);
        V fm[4];
        if (w[m] & kFvBnd) {
            // boundary face: its value at the face midpoint is one more data point
            const int bf = static_cast<int>(w[m] & ~kFvBnd);
            const T nx = FV_END_Y(m) - q[2 * m + 1], ny = -(FV_END_X(m) - q[2 * m]);  // outward
            fv_boundary_pairs<T>(G, bf, nx, ny, fc, f0, rho0, fm);
        } else {
            fv_load_row(sf, static_cast<int>(w[m] & 0xFFFFu), fm);
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const V df = PV::fma(fc[p], mone, fm[p]);  // f_m - f_c, one rounding
            gx[p] = PV::fma(wx, df, gx[p]);
            gy[p] = PV::fma(wy, df, gy[p]);
        }
    }
    // outgoing face values at every interior face: f_c + grad f_c . (x_f - x_c)
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (w[m] == kFvNone || (w[m] & kFvBnd)) continue;
        const V rx = PV::bcast(T(0.5) * (q[2 * m] + FV_END_X(m)));
        const V ry = PV::bcast(T(0.5) * (q[2 * m + 1] + FV_END_Y(m)));
        T out[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const V val = PV::fma(gy[p], ry, PV::fma(gx[p], rx, fc[p]));
            out[p] = ((w[m] >> (18 + p)) & 1u) ? val.x : val.y;
        }
        fv_store_vals(sv, c, m, out);
    }
}

// The same for one direction pair p of ring-1 cell c (four threads share a ring-1 cell, one
// pair each, and write one value per face slot each).
template <class T>
__device__ __forceinline__ void fv_cell_pair(int c, int p, const T *q, const T *lw, const uint4 &w4,
                                             const T *__restrict__ sf, const T *__restrict__ sf0,
                                             T *__restrict__ sv, const Geo<T> &G, T rho0) {
    using PV = FvPair<T>;
    using V = typename PV::V;
    const unsigned w[4] = {w4.x, w4.y, w4.z, w4.w};
    const V fc = *reinterpret_cast<const V *>(sf + fv_pair_off(c, p));
    const bool tri = w[3] == kFvNone;
    V gx = PV::bcast(T(0)), gy = PV::bcast(T(0));
    const V mone = PV::bcast(T(-1));
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (w[m] == kFvNone) continue;
        const V wx = PV::bcast(lw[2 * m]), wy = PV::bcast(lw[2 * m + 1]);
        V fm;
        if (w[m] & kFvBnd) {
            const int bf = static_cast<int>(w[m] & ~kFvBnd);
            const T nx = FV_END_Y(m) - q[2 * m + 1], ny = -(FV_END_X(m) - q[2 * m]);
            V fall[4], fb[4];
            fv_load_row(sf, c, fall);
            fv_boundary_pairs<T>(G, bf, nx, ny, fall, sf0[c], rho0, fb);
            fm = p == 0 ? fb[0] : (p == 1 ? fb[1] : (p == 2 ? fb[2] : fb[3]));
        } else {
            fm = *reinterpret_cast<const V *>(sf + fv_pair_off(static_cast<int>(w[m] & 0xFFFFu), p));
        }
        const V df = PV::fma(fc, mone, fm);
        gx = PV::fma(wx, df, gx);
        gy = PV::fma(wy, df, gy);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (w[m] == kFvNone || (w[m] & kFvBnd)) continue;
        const V rx = PV::bcast(T(0.5) * (q[2 * m] + FV_END_X(m)));
        const V ry = PV::bcast(T(0.5) * (q[2 * m + 1] + FV_END_Y(m)));
        const V val = PV::fma(gy, ry, PV::fma(gx, rx, fc));
        sv[fv_sv_off(c, m) + p] = ((w[m] >> (18 + p)) & 1u) ? val.x : val.y;
    }
}

// Convection term of item cell t (Eq. (advection)): per face its own outgoing values and the
// neighbour's (its incoming ones), both from the face-value rows, or the boundary values on a
// boundary face.  acc = sum_m (e_alpha . n_m dl_m / A) f_{alpha,bc,m} (= -Gamma^a).
template <class T>
__device__ __forceinline__ void fv_flux(int t, const T *q, const uint4 &wt, const T *fi,
                                        const T *__restrict__ sv, const Geo<T> &G, T rho0, T *acc) {
    using PV = FvPair<T>;
    using V = typename PV::V;
    const unsigned w[4] = {wt.x, wt.y, wt.z, wt.w};
    const bool tri = w[3] == kFvNone;
    T a2x = T(0);  // twice the area (shoelace on centroid-relative nodes)
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (m < 3 || !tri) a2x += q[2 * m] * FV_END_Y(m) - FV_END_X(m) * q[2 * m + 1];
    const T inv_a = a2x > T(0) ? sdiv(T(2), a2x) : T(0);  // padding cells have no faces
    V ac[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) ac[p] = PV::bcast(T(0));
    V fc[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) fc[p] = PV::make(fi[fv_first(p)], fi[fv_second(p)]);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (w[m] == kFvNone) continue;
        const T x1 = FV_END_X(m), y1 = FV_END_Y(m);
        const T snx = (y1 - q[2 * m + 1]) * inv_a;   // n dl / A
        const T sny = -(x1 - q[2 * m]) * inv_a;
        if (w[m] & kFvBnd) {
            const int bf = static_cast<int>(w[m] & ~kFvBnd);
            V fb[4];
            fv_boundary_pairs<T>(G, bf, snx, sny, fc, fi[0], rho0, fb);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const T en = fv_en<T>(p, snx, sny);
                ac[p] = PV::fma(PV::make(en, -en), fb[p], ac[p]);
            }
        } else {
            T vo[4], vn[4];
            fv_load_vals(sv, t, m, vo);
            fv_load_vals(sv, static_cast<int>(w[m] & 0xFFFFu), static_cast<int>((w[m] >> 16) & 3u), vn);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const T en = fv_en<T>(p, snx, sny);
                const bool out1 = (w[m] >> (18 + p)) & 1u;  // first member leaves here
                ac[p] = PV::fma(PV::make(en, -en), out1 ? PV::make(vo[p], vn[p]) : PV::make(vn[p], vo[p]),
                                ac[p]);
            }
        }
    }
    acc[0] = T(0);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        acc[fv_first(p)] = ac[p].x;
        acc[fv_second(p)] = ac[p].y;
    }
}

#undef FV_END_X
#undef FV_END_Y

// One IMEX stage (see fvlbm_kernels.cu's stage_algebra for what STAGE computes) in the
// face-value form, one CTA of 256 threads per work item.  fin: stage 1 f^n (structure of
// arrays), stages 2, 3 f^(2), f^(3) (cell-major rows); fs_out: stages 1, 2 write f^(2),
// f^(3) cell-major; fn: stage 3 writes f^{n+1}; geo: the cell-major geometry rows.
// In float, 3 CTAs per SM (80 registers, a few bytes spilled; 3 x 67 KB of shared memory)
// run the sweep 4 % faster than 2 CTAs with 105 registers: the stages are latency-bound.
template <class T, int STAGE, bool STATS>
__global__ void __launch_bounds__(kFvThreads, sizeof(T) == 4 ? 3 : 1)
    k_fused_fv(const T *__restrict__ fin, T *__restrict__ fs_out, T *__restrict__ fn,
               T *__restrict__ Bacc, T *__restrict__ Cacc, const T *__restrict__ tau,
               T *__restrict__ mac, double *__restrict__ partial, Geo<T> G, FvItems W,
               const T *__restrict__ geo) {
    using PV = FvPair<T>;
    using V = typename PV::V;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sf = reinterpret_cast<T *>(smem_raw + FvSmem<T>::sf);
    T *sf0 = reinterpret_cast<T *>(smem_raw + FvSmem<T>::sf0);
    T *stau = reinterpret_cast<T *>(smem_raw + FvSmem<T>::st);
    T *sdt = stau + kFvEcap;
    T *sv = reinterpret_cast<T *>(smem_raw + FvSmem<T>::sv);
    uint4 *sa = reinterpret_cast<uint4 *>(smem_raw + FvSmem<T>::sa);
    T *sacc = reinterpret_cast<T *>(smem_raw + FvSmem<T>::sacc);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + FvSmem<T>::bar);

    const int t = threadIdx.x;
    const int it = W.item0 + static_cast<int>(blockIdx.x);
    // halo slot t of the fixed-stride table and the header, loaded together (kept in L2)
    const unsigned long long keep = l2_keep_policy();
    const int gid0 = t < kFvHs ? ld_keep(W.halo + static_cast<size_t>(it) * kFvHs + t, keep) : -1;
    const int4 hd = ld_keep(W.hdr + it, keep);
    const int base = hd.x, cnt = hd.y & 0xFFFF, nr1 = hd.y >> 16;
    const int NG = cnt + nr1;
    // slot kFvHs + t, in the overflow table (items split for their large halo only)
    const int gid1 = hd.w >= 0 && t < kFvHs ? ld_keep(W.ovf + hd.w + t, keep) : -1;
    const uint4 *__restrict__ adj_g = W.adj + static_cast<size_t>(it) * kFvGcap;
    const size_t np = G.np;
    const InstParam *__restrict__ Pp = G.ip + hd.z;  // read where used
    const T rho0 = ipv<T>(Pp->rho0, Pp->rho0_f);
    const bool mine = t < cnt;
    const int i = base + t;
    const T *fa0 = fin + 8 * np;  // stages 2, 3: f_0 of every cell after the cell-major rows

    // 1. staging, issued before any wait
    // The bulk copies are shared out over the lanes 0 of the 8 warps, so that no warp issues
    // more than 3 of them: each such lane arrives on the mbarrier (count 8) with the bytes of
    // its own copies, then issues them.
    constexpr int kWarps = kFvThreads / 32;
    if (t == 0) mbar_init(bar, kWarps);
    __syncthreads();
    if ((t & 31) == 0) {
        const unsigned row = static_cast<unsigned>(cnt * sizeof(T));
        // copies: (stages 2, 3) the item's f rows and f_0, then the accumulator rows (stage 1:
        // f^n, stage 2: B and C, stage 3: C), then tau
        const T *a1g = STAGE == 1 ? fin : (STAGE == 2 ? Bacc : Cacc);
        constexpr int nf = STAGE == 1 ? 0 : 2, nacc = STAGE == 2 ? 2 * kQ : kQ, ncopy = nf + nacc + 1;
        const int w = t >> 5;
        unsigned bytes = 0;
        for (int c = w; c < ncopy; c += kWarps) bytes += (nf > 0 && c == 0) ? 8 * row : row;
        mbar_expect_tx(bar, bytes);
        for (int c = w; c < ncopy; c += kWarps) {
            if (nf > 0 && c == 0) {
                bulk_g2s(sf, fin + 8 * static_cast<size_t>(base), 8 * row, bar);
            } else if (nf > 0 && c == 1) {
                bulk_g2s(sf0, fa0 + base, row, bar);
            } else if (c < nf + kQ) {
                const int a = c - nf;
                bulk_g2s(sacc + a * kFvThreads, a1g + a * np + base, row, bar);
            } else if (c < nf + nacc) {  // stage 2: the C rows
                const int a = c - nf - kQ;
                bulk_g2s(sacc + (kQ + a) * kFvThreads, Cacc + a * np + base, row, bar);
            } else {
                bulk_g2s(sacc + 2 * kQ * kFvThreads, tau + base, row, bar);
            }
        }
    }
    constexpr int per = 16 / sizeof(T);  // elements per 16-byte chunk
#pragma unroll
    for (int k = 0; k < 2; ++k) {  // halo cells (item rows come in bulk): slots t, kFvHs + t
        const int gid = k == 0 ? gid0 : gid1;
        if (gid < 0) continue;
        const int e = cnt + t + k * kFvHs;
        if (STAGE == 1) {  // f^n is structure of arrays: one element per direction
#pragma unroll
            for (int a = 1; a < kQ; ++a) cp_async<sizeof(T)>(sf + fv_alpha_off(e, a), fin + a * np + gid);
            cp_async<sizeof(T)>(sf0 + e, fin + gid);
            cp_async<sizeof(T)>(stau + e, tau + gid);
            if (G.dtc != nullptr) cp_async<sizeof(T)>(sdt + e, G.dtc + gid);
        } else {  // one cell-major row: half h sits at half fv_half(gid, h) there, fv_half(e, h) here
            const T *src = fin + 8 * static_cast<size_t>(gid);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int k = 0; k < 4 / per; ++k)
                    cp_async<16>(sf + e * 8 + 4 * fv_half(e, h) + k * per, src + 4 * fv_half(gid, h) + k * per);
            cp_async<sizeof(T)>(sf0 + e, fa0 + gid);
        }
        if (e < NG) {  // ring-1 geometry into its face-value row (swizzled 16-byte chunks)
            const T *g = geo + 16 * static_cast<size_t>(gid);
            const int cs = (e >> 1) & 3;
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int h = 0; h < 4 / per; ++h)
                    cp_async<16>(sv + e * 16 + 4 * (k ^ cs) + h * per, g + 4 * k + h * per);
        }
    }
    for (int e = t; e < NG; e += kFvThreads) cp_async<16>(sa + e, adj_g + e);
    static_assert(sizeof(InstParam) % 16 == 0 && FvSmem<T>::ip % 16 == 0, "16-byte copies of the parameters");
    if (t < static_cast<int>(sizeof(InstParam) / 16))  // (device arrays of InstParam: 16-byte aligned rows)
        cp_async<16>(smem_raw + FvSmem<T>::ip + 16 * t, reinterpret_cast<const unsigned char *>(Pp) + 16 * t);
    T q[8], lw[8];
    if (mine) fv_load_geo_row(geo + 16 * static_cast<size_t>(i), q, lw);  // the item cell's geometry row
    cp_async_wait_all();
    // stage 1: each thread relaxes the halo cells it staged (its own copies have landed)
    const T dtg = ipv<T>(Pp->dt, Pp->dt_f);
    if (STAGE == 1) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if ((k == 0 ? gid0 : gid1) < 0) continue;
            const int e = cnt + t + k * kFvHs;
            T f[kQ];
            f[0] = sf0[e];
#pragma unroll
            for (int a = 1; a < kQ; ++a) f[a] = sf[fv_alpha_off(e, a)];
            fv_relax_to_row(f, sf, sf0, e, rho0, G.dtc != nullptr ? sdt[e] : dtg, stau[e]);
        }
    }
    {
        long long it = 0;
        // (a limit of 0 gives up at once, without polling: the diagnostic of the error path)
        bool done = W.wait_first > 0 && mbar_try_wait(bar, 0);
        while (!done && ++it < W.wait_first) done = mbar_try_wait(bar, 0);
        // the block leaves together if any thread gave up: flag it, wait once more (with the
        // full bound) for its own copies in flight, then return
        if (__syncthreads_or(!done)) {
            if (t == 0) atomicExch(W.err, 1);
            for (long long k = 0; k < kWaitLimit && !mbar_try_wait(bar, 0); ++k) {
            }
            return;
        }
    }
    // stage 1: the item cells' f^(1) from their f^n rows (in the accumulator copy)
    if (STAGE == 1 && mine) {
        T f[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) f[a] = sacc[a * kFvThreads + t];
        // its f^eq(f^n) goes to the free accumulator rows kQ.. (stage 1 copies no C rows), where
        // the stage-1 algebra reads it instead of forming it again
        T eq[kQ];
        fv_relax_to_row(f, sf, sf0, t, rho0, G.dtc != nullptr ? G.dtc[i] : dtg, sacc[2 * kQ * kFvThreads + t], eq);
#pragma unroll
        for (int a = 0; a < kQ; ++a) sacc[(kQ + a) * kFvThreads + t] = eq[a];
    }
    // ring-1 geometry for the pair-split work below, read before any face value is written
    const int ru = 4 * nr1;  // ring-1 work units: (cell, pair)
    T qr[8], lr[8];
    uint4 wr = make_uint4(kFvNone, kFvNone, kFvNone, kFvNone);
    if (t < ru) {
        const int c = cnt + (t >> 2);
        fv_load_vals(sv, c, 0, qr);
        fv_load_vals(sv, c, 1, qr + 4);
        fv_load_vals(sv, c, 2, lr);
        fv_load_vals(sv, c, 3, lr + 4);
        wr = sa[c];
    }
    __syncthreads();

    // 2. gradients and outgoing face values: item cells (thread t takes cell t), then ring-1
    //    cells with one direction pair per thread
    if (mine) fv_cell<T>(t, q, lw, sa[t], sf, sf0[t], sv, G, rho0);
    if (t < ru) fv_cell_pair<T>(cnt + (t >> 2), t & 3, qr, lr, wr, sf, sf0, sv, G, rho0);
    // items with more than 64 ring-1 cells: further rounds of 256 units.  A ring-1 row is
    // written only by the four threads of its own unit (consecutive lanes of one warp) in its
    // own round, so each thread reads the geometry from its row and the warp syncs before any
    // of them writes a face value there.  The round count is the same for the whole block.
    for (int u0 = kFvThreads; u0 < ru; u0 += kFvThreads) {
        const int u = u0 + t;
        const bool act = u < ru;
        const int c = cnt + (u >> 2);
        T q2[8], l2[8];
        if (act) {
            fv_load_vals(sv, c, 0, q2);
            fv_load_vals(sv, c, 1, q2 + 4);
            fv_load_vals(sv, c, 2, l2);
            fv_load_vals(sv, c, 3, l2 + 4);
        }
        __syncwarp();
        if (act) fv_cell_pair<T>(c, u & 3, q2, l2, sa[c], sf, sf0, sv, G, rho0);
    }
    __syncthreads();

    // 3. flux of item cell t (Eq. (advection)) from the published face values
    double st[4] = {0.0, 0.0, 0.0, 0.0};
    if (mine) {
        T fi[kQ], acc[kQ];
        const uint4 wt = sa[t];
        V fr[4];
        fv_load_row(sf, t, fr);
        fi[0] = sf0[t];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            fi[fv_first(p)] = fr[p].x;
            fi[fv_second(p)] = fr[p].y;
        }
        fv_flux<T>(t, q, wt, fi, sv, G, rho0, acc);

        // 4. the stage algebra, with the accumulator rows, tau and the parameters from shared memory
        const InstParam &P = *reinterpret_cast<const InstParam *>(smem_raw + FvSmem<T>::ip);
        T macv[3];
        T uo = T(0), vo0 = T(0);
        if (STATS) {
            uo = mac[1 * np + i];
            vo0 = mac[2 * np + i];
        }
        const T tau_i = sacc[2 * kQ * kFvThreads + t];
        stage_algebra<T, STAGE, false, kFvThreads, false, true, STAGE == 1>(
            i, np, fi, acc, P, tau_i, cell_dt(G, P, i), sacc, kFvThreads, t, sacc + kQ * kFvThreads, kFvThreads,
            t, fs_out, fn, Bacc, Cacc, mac, nullptr, G.area, nullptr, false, T(0), macv);
        if (STATS) {
            const double un = double(macv[1]), vn = double(macv[2]), r = double(macv[0]);
            const bool bad = !(isfinite(un) && isfinite(vn) && isfinite(r));
            st[0] = (un - double(uo)) * (un - double(uo)) + (vn - double(vo0)) * (vn - double(vo0));
            st[1] = un * un + vn * vn;
            st[2] = r * double(G.area[i]);
            st[3] = bad ? 1.0 : 0.0;
        }
    }
    if (STATS) block_sum<4, kFvThreads>(st, partial + 4 * it);
}
