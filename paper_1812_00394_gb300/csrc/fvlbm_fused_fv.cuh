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
// Staging uses cp.async only (no mbarrier wait, so nothing can spin), all issued at the start
// and waited for once: f^(J) of the item, ring-1 and ring-2 cells in pair-ordered rows, the
// geometry and adjacency of item and ring-1 cells, and the item's accumulator rows and tau, so
// that no phase after the wait touches global memory except for its stores.
// Stage 1 stages f^n with tau and relaxes every staged cell to f^(1) on chip, so no f^(1)
// array passes through HBM between steps (and f^n is never recovered from a rounded f^(1)).
//
// FP32 arithmetic runs on packed pairs (fma.rn.f32x2): the two members of a pair share every
// geometric factor, so the gradient and face-value updates are one packed FMA per pair.

// Shared-memory capacity of the face-value kernel (cells): ring-1 + ring-2 + item cells and
// item + ring-1 cells.  256-cell blocks whose halo exceeds it are split.
// Cells per work item (and threads per CTA): 256, or 128 with proportionally smaller halos.
#ifndef FVLBM_FV_ITEM
#define FVLBM_FV_ITEM 256
#endif
constexpr int kFvThreads = FVLBM_FV_ITEM;
constexpr int kFvEcap = FVLBM_FV_ITEM == 256 ? 448 : 256;
constexpr int kFvGcap = FVLBM_FV_ITEM == 256 ? 352 : 192;
// CTAs per SM the FP32 kernel is compiled for (registers per thread: 128 at 2 CTAs of 256)
#ifndef FVLBM_FV_MIN_BLOCKS
#define FVLBM_FV_MIN_BLOCKS (512 / FVLBM_FV_ITEM)
#endif

// Adjacency word of the face-value kernel (cell-major: 4 words per cell):
//   0xFFFFFFFF: no face; bit 31 set: boundary face (low 31 bits: global boundary face index);
//   else: local index (bits 0-15) | back slot (16-17) | outgoing bits (18-21), bit 18 + p set
//   when the first member of pair p leaves this cell through the face.
constexpr unsigned kFvNone = 0xFFFFFFFFu;
constexpr unsigned kFvBnd = 0x80000000u;

struct FvItems {
    const int4 *__restrict__ hdr;       // [nitem + 1]: base cell, cells, halo offset, adj offset
    const int *__restrict__ r1;         // [nitem] ring-1 count
    const int *__restrict__ halo;       // global ids: ring 1 then ring 2, per item
    const uint4 *__restrict__ adj;      // per item [cells + r1] adjacency (cell-major)
    int *__restrict__ err;              // set to 1 if the bulk-copy wait gave up
    long long wait_first;               // polls of that wait (fvlbm_set_wait_limit)
};

// Pair p: first members alpha = 1, 2, 5, 6 and their opposites 3, 4, 7, 8.
__host__ __device__ constexpr int fv_first(int p) { return p == 0 ? 1 : (p == 1 ? 2 : (p == 2 ? 5 : 6)); }
__host__ __device__ constexpr int fv_second(int p) { return p == 0 ? 3 : (p == 1 ? 4 : (p == 2 ? 7 : 8)); }

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

// Shared-memory layout (elements of T):
//   sf  [kFvEcap][8]   f^(J), alpha = 1..8 in pair order (1,3)(2,4)(5,7)(6,8); the two 4-value
//                      halves of row j are swapped when bit 2 of j is set (bank spread)
//   sf0 [kFvEcap]      f^(J)_0 of item, ring-1 and ring-2 cells
//   st  [2][kFvEcap]   tau of the staged cells (stage 1: every staged cell, to relax f^n to
//                      f^(1) in place with Eq. (fnewstage), J = 1; stages 2, 3: item cells),
//                      and in stage 1 the cells' time steps under local time stepping
//   sv  [kFvGcap][16]  outgoing face values, 4 per face slot; 16-byte chunk m of row c sits at
//                      chunk m ^ ((c >> 1) & 3).  Before the face values are written, the
//                      rows of ring-1 cells hold their geometry in the same swizzled chunks:
//                      node offsets q[0..3], q[4..7], least-squares weights W[0..3], W[4..7]
//   sa  [kFvGcap]      adjacency words (uint4)
//   sacc [18][256]     the item's accumulator rows for the stage algebra, SoA (stage 1: f^n;
//                      stage 2: B and C; stage 3: C), by bulk copy
//   one mbarrier for the bulk copies
template <class T>
struct FvSmem {
    static constexpr size_t sf = 0;
    static constexpr size_t sf0 = sf + size_t(kFvEcap) * 8 * sizeof(T);
    static constexpr size_t st = sf0 + ((size_t(kFvEcap) * sizeof(T) + 15) / 16) * 16;
    static constexpr size_t sv = st + 2 * size_t(kFvEcap) * sizeof(T);
    static constexpr size_t sa = sv + size_t(kFvGcap) * 16 * sizeof(T);
    static constexpr size_t sacc = sa + size_t(kFvGcap) * 16;
    static constexpr size_t bar = sacc + size_t(18) * kFvThreads * sizeof(T);
    static constexpr size_t bytes = bar + 16;
};

// Position of alpha (1..8) within a pair-ordered row of 8: (1,3)(2,4)(5,7)(6,8).
__host__ __device__ constexpr int fv_pos(int a) {
    return a == 1 ? 0 : (a == 3 ? 1 : (a == 2 ? 2 : (a == 4 ? 3 : (a == 5 ? 4 : (a == 7 ? 5 : (a == 6 ? 6 : 7))))));
}
// element offset of face slot m in row c of sv
__device__ __forceinline__ int fv_sv_off(int c, int m) { return c * 16 + 4 * (m ^ ((c >> 1) & 3)); }

// Load the 8 moving directions of row j as 4 pairs.
template <class T>
__device__ __forceinline__ void fv_load_row(const T *sf, int j, typename FvPair<T>::V *o) {
    using PV = FvPair<T>;
    const int sw = (j & 4) ? 4 : 0;
    const T *row = sf + j * 8;
    if constexpr (sizeof(T) == 4) {
        const float4 lo = *reinterpret_cast<const float4 *>(row + sw);
        const float4 hi = *reinterpret_cast<const float4 *>(row + (sw ^ 4));
        o[0] = PV::make(lo.x, lo.y);
        o[1] = PV::make(lo.z, lo.w);
        o[2] = PV::make(hi.x, hi.y);
        o[3] = PV::make(hi.z, hi.w);
    } else {
        const double2 a = *reinterpret_cast<const double2 *>(row + sw);
        const double2 b = *reinterpret_cast<const double2 *>(row + sw + 2);
        const double2 c = *reinterpret_cast<const double2 *>(row + (sw ^ 4));
        const double2 d = *reinterpret_cast<const double2 *>(row + (sw ^ 4) + 2);
        o[0] = a;
        o[1] = b;
        o[2] = c;
        o[3] = d;
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

// Boundary face values (boundary_values) of a cell whose f is given as 4 pairs and f_0, as 4
// pairs.
template <class T>
__device__ __forceinline__ void fv_boundary_pairs(int type, const T *__restrict__ bval, int nbt, T nx, T ny,
                                               const typename FvPair<T>::V *fc, T f0, T rho0,
                                               typename FvPair<T>::V *out) {
    using PV = FvPair<T>;
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
// of staged cell e, in place.
template <class T>
__device__ __forceinline__ void fv_relax_row(T *sf, T *sf0, int e, T rho0, T dt, T tau_e) {
    using V = typename FvPair<T>::V;
    V fr[4];
    fv_load_row(sf, e, fr);
    T f[kQ];
    f[0] = sf0[e];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        f[fv_first(p)] = fr[p].x;
        f[fv_second(p)] = fr[p].y;
    }
    relax9(f, rho0, dt, tau_e);
    sf0[e] = f[0];
    const int sw = (e & 4) ? 4 : 0;
#pragma unroll
    for (int a = 1; a < kQ; ++a) sf[e * 8 + (fv_pos(a) ^ sw)] = f[a];
}

// Gradient (Step 2) and outgoing face values of item / ring-1 cell c.  q: node positions
// relative to the centroid; lw: least-squares weights W_m = M^{-1} d_m (x, y per face slot);
// w: adjacency.
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
    // end node of face m (m compile-time): node m + 1, wrapping to node 0 after the last face;
    // selects between static indices keep q in registers
    auto end_x = [&](int m) { return m == 3 ? q[0] : (m == 2 && tri ? q[0] : q[2 * m + 2]); };
    auto end_y = [&](int m) { return m == 3 ? q[1] : (m == 2 && tri ? q[1] : q[2 * m + 3]); };
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
            const T nx = end_y(m) - q[2 * m + 1], ny = -(end_x(m) - q[2 * m]);  // outward (unscaled)
            fv_boundary_pairs<T>(G.btype[bf], G.bval + bf, G.nbt, nx, ny, fc, f0, rho0, fm);
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
        const V rx = PV::bcast(T(0.5) * (q[2 * m] + end_x(m)));
        const V ry = PV::bcast(T(0.5) * (q[2 * m + 1] + end_y(m)));
        T out[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const V val = PV::fma(gy[p], ry, PV::fma(gx[p], rx, fc[p]));
            out[p] = ((w[m] >> (18 + p)) & 1u) ? val.x : val.y;
        }
        fv_store_vals(sv, c, m, out);
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
    auto end_x = [&](int m) { return m == 3 ? q[0] : (m == 2 && tri ? q[0] : q[2 * m + 2]); };
    auto end_y = [&](int m) { return m == 3 ? q[1] : (m == 2 && tri ? q[1] : q[2 * m + 3]); };
    T a2x = T(0);  // twice the area (shoelace on centroid-relative nodes)
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (m < 3 || !tri) a2x += q[2 * m] * end_y(m) - end_x(m) * q[2 * m + 1];
    const T inv_a = a2x > T(0) ? T(2) / a2x : T(0);  // padding cells have no faces
    V ac[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) ac[p] = PV::bcast(T(0));
    V fc[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) fc[p] = PV::make(fi[fv_first(p)], fi[fv_second(p)]);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (w[m] == kFvNone) continue;
        const T x1 = end_x(m), y1 = end_y(m);
        const T snx = (y1 - q[2 * m + 1]) * inv_a;   // n dl / A
        const T sny = -(x1 - q[2 * m]) * inv_a;
        if (w[m] & kFvBnd) {
            const int bf = static_cast<int>(w[m] & ~kFvBnd);
            V fb[4];
            fv_boundary_pairs<T>(G.btype[bf], G.bval + bf, G.nbt, snx, sny, fc, fi[0], rho0, fb);
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

// One IMEX stage (see fvlbm_kernels.cu's stage_algebra for what STAGE computes) in the
// face-value form, one CTA of 256 threads per work item.
template <class T, int STAGE, bool STATS>
__global__ void __launch_bounds__(kFvThreads, sizeof(T) == 4 ? FVLBM_FV_MIN_BLOCKS : 1)
    k_fused_fv(const T *__restrict__ fin, T *__restrict__ fs_out, T *__restrict__ fn,
               T *__restrict__ Bacc, T *__restrict__ Cacc, const T *__restrict__ tau,
               T *__restrict__ mac, double *__restrict__ partial, Geo<T> G, FvItems W,
               T *__restrict__ frel, CompactGeo<T> CG) {
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
    const int4 hd = W.hdr[blockIdx.x];
    const int base = hd.x, cnt = hd.y, h0 = hd.z;
    const int nh = W.hdr[blockIdx.x + 1].z - h0;
    const int nr1 = W.r1[blockIdx.x];
    const int E = cnt + nh, NG = cnt + nr1;
    const uint4 *__restrict__ adj_g = W.adj + hd.w;
    const size_t np = G.np;
    const InstParam *__restrict__ Pp = G.ip + G.tile_inst[base / kTile];  // read where used
    const T rho0 = ipv<T>(Pp->rho0, Pp->rho0_f);
    const bool mine = t < cnt;
    const int i = base + t;

    // 1. staging, issued before any wait: the item's accumulator rows (and tau) by bulk copies
    //    on one mbarrier; f^(J) of item, ring-1 and ring-2 cells, the adjacency and the ring-1
    //    geometry by cp.async; the item cell's own geometry straight into registers
    if (t == 0) mbar_init(bar);
    __syncthreads();
    if (t == 0) {
        const unsigned row = static_cast<unsigned>(cnt * sizeof(T));
        const int nrows = STAGE == 2 ? 2 * kQ : kQ;
        mbar_expect_tx(bar, row * (nrows + (STAGE == 1 ? 0 : 1)));
        const T *a1g = STAGE == 1 ? fin : (STAGE == 2 ? Bacc : Cacc);
        for (int a = 0; a < kQ; ++a) bulk_g2s(sacc + a * kFvThreads, a1g + a * np + base, row, bar);
        if (STAGE == 2)
            for (int a = 0; a < kQ; ++a) bulk_g2s(sacc + (kQ + a) * kFvThreads, Cacc + a * np + base, row, bar);
        if (STAGE != 1) bulk_g2s(stau, tau + base, row, bar);
    }
    for (int e = t; e < E; e += kFvThreads) {
        const int gid = e < cnt ? base + e : W.halo[h0 + e - cnt];
        const int sw = (e & 4) ? 4 : 0;
#pragma unroll
        for (int a = 1; a < kQ; ++a)
            cp_async<sizeof(T)>(sf + e * 8 + (fv_pos(a) ^ sw), fin + a * np + gid);
        cp_async<sizeof(T)>(sf0 + e, fin + gid);
        if (STAGE == 1) {
            cp_async<sizeof(T)>(stau + e, tau + gid);
            if (G.dtc != nullptr) cp_async<sizeof(T)>(sdt + e, G.dtc + gid);
        }
        if (e < NG) {
            cp_async<16>(sa + e, adj_g + e);
            if (e >= cnt) {  // ring-1 geometry into its face-value row (swizzled 16-byte chunks)
                const int cs = (e >> 1) & 3;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    cp_async<sizeof(T)>(sv + e * 16 + 4 * ((k >> 2) ^ cs) + (k & 3), CG.gq + k * np + gid);
                    cp_async<sizeof(T)>(sv + e * 16 + 4 * ((2 + (k >> 2)) ^ cs) + (k & 3), G.lsq + k * np + gid);
                }
            }
        }
    }
    T q[8], lw[8];
    if (mine) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            q[k] = CG.gq[k * np + i];
            lw[k] = G.lsq[k * np + i];
        }
    }
    cp_async_wait_all();
    // stage 1: each thread relaxes the cells it staged itself (its own copies have landed), so
    // the relaxation needs no barrier of its own
    if (STAGE == 1) {
        const T dtg = ipv<T>(Pp->dt, Pp->dt_f);
        for (int e = t; e < E; e += kFvThreads)
            fv_relax_row(sf, sf0, e, rho0, G.dtc != nullptr ? sdt[e] : dtg, stau[e]);
    }
    {
        long long it = 0;
        // (a limit of 0 polls once without blocking: try_wait itself may suspend the thread for
        // a while, test_wait returns at once)
        bool done = W.wait_first > 0 ? mbar_try_wait(bar, 0) : mbar_test_wait(bar, 0);
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

    // 2. gradients and outgoing face values of item and ring-1 cells
    if (mine) fv_cell<T>(t, q, lw, sa[t], sf, sf0[t], sv, G, rho0);
    for (int c = (mine ? t + kFvThreads : t); c < NG; c += kFvThreads) {
        if (c < cnt) continue;  // only when cnt < 256: item cells are all handled above
        T qr[8], lr[8];
        fv_load_vals(sv, c, 0, qr);       // geometry chunks staged in the face-value row
        fv_load_vals(sv, c, 1, qr + 4);
        fv_load_vals(sv, c, 2, lr);
        fv_load_vals(sv, c, 3, lr + 4);
        fv_cell<T>(c, qr, lr, sa[c], sf, sf0[c], sv, G, rho0);
    }
    __syncthreads();

    // 3. flux of item cell t (Eq. (advection)) from the published face values
    T fi[kQ], acc[kQ];
    double st[4] = {0.0, 0.0, 0.0, 0.0};
    if (mine) {
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

        // 4. the stage algebra, with the accumulator rows and tau from shared memory
        const InstParam P = *Pp;
        T macv[3];
        T uo = T(0), vo0 = T(0);
        if (STATS) {
            uo = mac[1 * np + i];
            vo0 = mac[2 * np + i];
        }
        stage_algebra<T, STAGE, false, kFvThreads, false>(i, np, fi, acc, P, stau[t], cell_dt(G, P, i), sacc,
                                                          kFvThreads, t, sacc + kQ * kFvThreads, kFvThreads, t,
                                                          fs_out, fn, Bacc, Cacc, mac, nullptr, G.area, frel,
                                                          false, T(0), macv);
        if (STATS) {
            const double un = double(macv[1]), vn = double(macv[2]), r = double(macv[0]);
            const bool bad = !(isfinite(un) && isfinite(vn) && isfinite(r));
            st[0] = (un - double(uo)) * (un - double(uo)) + (vn - double(vo0)) * (vn - double(vo0));
            st[1] = un * un + vn * vn;
            st[2] = r * double(G.area[i]);
            st[3] = bad ? 1.0 : 0.0;
        }
    }
    if (STATS) block_sum<4, kFvThreads>(st, partial + 4 * blockIdx.x);
}

// ------------------------------------------------------------------ persistent form
// The same stage in a persistent kernel: a grid of (SMs x resident CTAs) walks the work items
// round-robin (CTA b takes items b, b + grid, b + 2 grid, ...: at any time the grid works on a
// window of consecutive items, whose halos are each other's cells and stay in L2).  While a
// CTA computes item k, the copies of item k+1 are in flight:
//   - f^(J) of its item, ring-1 and ring-2 cells, its adjacency, the ring-1 geometry (and in
//     stage 1 tau and dt of every staged cell) go into the second of two staging buffers by
//     cp.async, issued when item k starts;
//   - its accumulator rows and tau (bulk copies on one mbarrier) and its cells' own geometry
//     (cp.async into their face-value rows) are issued when item k has finished with them.
// Only the face-value rows and the accumulator rows are single-buffered.

constexpr int kFvR1cap = 96;   // ring-1 cells of one item (the host splits items beyond it)

template <class T>
struct FvpSmem {
    // one staging buffer
    static constexpr size_t sf = 0;
    static constexpr size_t sf0 = sf + size_t(kFvEcap) * 8 * sizeof(T);
    static constexpr size_t st = sf0 + ((size_t(kFvEcap) * sizeof(T) + 15) / 16) * 16;
    static constexpr size_t sa = st + 2 * size_t(kFvEcap) * sizeof(T);
    static constexpr size_t sg = sa + size_t(kFvGcap) * 16;
    static constexpr size_t buf = sg + size_t(kFvR1cap) * 16 * sizeof(T);
    // shared by the items
    static constexpr size_t sv = 2 * buf;
    static constexpr size_t sacc = sv + size_t(kFvGcap) * 16 * sizeof(T);
    static constexpr size_t bar = sacc + size_t(2 * kQ + 1) * kFvThreads * sizeof(T);
    static constexpr size_t bytes = bar + 16;
};

struct FvItem {
    int base, cnt, h0, nh, nr1, adj0;
};

__device__ __forceinline__ FvItem fv_item(const FvItems &W, int k) {
    const int4 hd = W.hdr[k];
    FvItem it;
    it.base = hd.x;
    it.cnt = hd.y;
    it.h0 = hd.z;
    it.nh = W.hdr[k + 1].z - hd.z;
    it.nr1 = W.r1[k];
    it.adj0 = hd.w;
    return it;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// cp.async of the staging buffer of one item (f^(J) of item, ring-1 and ring-2 cells; stage 1:
// tau and dt of each; adjacency of item and ring-1 cells; ring-1 geometry)
template <class T, int STAGE>
__device__ __forceinline__ void fvp_stage_buffer(unsigned char *b, const FvItem &it, const T *__restrict__ fin,
                                                 const T *__restrict__ tau, const FvItems &W,
                                                 const Geo<T> &G, const CompactGeo<T> &CG) {
    T *sf = reinterpret_cast<T *>(b + FvpSmem<T>::sf);
    T *sf0 = reinterpret_cast<T *>(b + FvpSmem<T>::sf0);
    T *stau = reinterpret_cast<T *>(b + FvpSmem<T>::st);
    T *sdt = stau + kFvEcap;
    uint4 *sa = reinterpret_cast<uint4 *>(b + FvpSmem<T>::sa);
    T *sg = reinterpret_cast<T *>(b + FvpSmem<T>::sg);
    const size_t np = G.np;
    const int E = it.cnt + it.nh, NG = it.cnt + it.nr1;
    for (int e = threadIdx.x; e < E; e += kFvThreads) {
        const int gid = e < it.cnt ? it.base + e : W.halo[it.h0 + e - it.cnt];
        const int sw = (e & 4) ? 4 : 0;
#pragma unroll
        for (int a = 1; a < kQ; ++a)
            cp_async<sizeof(T)>(sf + e * 8 + (fv_pos(a) ^ sw), fin + a * np + gid);
        cp_async<sizeof(T)>(sf0 + e, fin + gid);
        if (STAGE == 1) {
            cp_async<sizeof(T)>(stau + e, tau + gid);
            if (G.dtc != nullptr) cp_async<sizeof(T)>(sdt + e, G.dtc + gid);
        }
        if (e < NG) {
            cp_async<16>(sa + e, W.adj + it.adj0 + e);
            if (e >= it.cnt) {  // ring-1 geometry, swizzled 16-byte chunks like the face values
                const int r = e - it.cnt, cs = (e >> 1) & 3;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    cp_async<sizeof(T)>(sg + r * 16 + 4 * ((k >> 2) ^ cs) + (k & 3), CG.gq + k * np + gid);
                    cp_async<sizeof(T)>(sg + r * 16 + 4 * ((2 + (k >> 2)) ^ cs) + (k & 3), G.lsq + k * np + gid);
                }
            }
        }
    }
}

// Copies of one item issued once the previous item has finished with the single buffers:
// the item cells' geometry into their face-value rows (cp.async) and, by thread 0, the
// accumulator rows and tau (bulk copies on the mbarrier).
template <class T, int STAGE>
__device__ __forceinline__ void fvp_stage_item_rows(const FvItem &it, T *sv, T *sacc, unsigned long long *bar,
                                                    const T *__restrict__ fin, const T *__restrict__ Bacc,
                                                    const T *__restrict__ Cacc, const T *__restrict__ tau,
                                                    const Geo<T> &G, const CompactGeo<T> &CG) {
    const size_t np = G.np;
    const int e = threadIdx.x;
    if (e < it.cnt) {
        const int gid = it.base + e, cs = (e >> 1) & 3;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            cp_async<sizeof(T)>(sv + e * 16 + 4 * ((k >> 2) ^ cs) + (k & 3), CG.gq + k * np + gid);
            cp_async<sizeof(T)>(sv + e * 16 + 4 * ((2 + (k >> 2)) ^ cs) + (k & 3), G.lsq + k * np + gid);
        }
    }
    if (e == 0) {
        const unsigned row = static_cast<unsigned>(it.cnt * sizeof(T));
        const int nrows = (STAGE == 2 ? 2 * kQ : kQ) + (STAGE == 1 ? 0 : 1);
        mbar_expect_tx(bar, row * nrows);
        const T *a1g = STAGE == 1 ? fin : (STAGE == 2 ? Bacc : Cacc);
        for (int a = 0; a < kQ; ++a) bulk_g2s(sacc + a * kFvThreads, a1g + a * np + it.base, row, bar);
        if (STAGE == 2)
            for (int a = 0; a < kQ; ++a)
                bulk_g2s(sacc + (kQ + a) * kFvThreads, Cacc + a * np + it.base, row, bar);
        if (STAGE != 1) bulk_g2s(sacc + 2 * kQ * kFvThreads, tau + it.base, row, bar);
    }
}

template <class T, int STAGE, bool STATS>
__global__ void __launch_bounds__(kFvThreads, sizeof(T) == 4 ? 2 : 1)
    k_fused_fvp(const T *__restrict__ fin, T *__restrict__ fs_out, T *__restrict__ fn,
                T *__restrict__ Bacc, T *__restrict__ Cacc, const T *__restrict__ tau,
                T *__restrict__ mac, double *__restrict__ partial, Geo<T> G, FvItems W,
                CompactGeo<T> CG, int nitem) {
    using PV = FvPair<T>;
    using V = typename PV::V;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sv = reinterpret_cast<T *>(smem_raw + FvpSmem<T>::sv);
    T *sacc = reinterpret_cast<T *>(smem_raw + FvpSmem<T>::sacc);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + FvpSmem<T>::bar);
    const int t = threadIdx.x;
    const size_t np = G.np;

    int k = blockIdx.x;
    if (k >= nitem) return;
    if (t == 0) mbar_init(bar);
    __syncthreads();
    // prologue: the first item's copies
    FvItem it = fv_item(W, k);
    fvp_stage_buffer<T, STAGE>(smem_raw, it, fin, tau, W, G, CG);
    fvp_stage_item_rows<T, STAGE>(it, sv, sacc, bar, fin, Bacc, Cacc, tau, G, CG);
    cp_async_commit();
    unsigned phase = 0;
    for (int p = 0; k < nitem; k += gridDim.x, p ^= 1, phase ^= 1) {
        unsigned char *b = smem_raw + p * FvpSmem<T>::buf;
        T *sf = reinterpret_cast<T *>(b + FvpSmem<T>::sf);
        T *sf0 = reinterpret_cast<T *>(b + FvpSmem<T>::sf0);
        T *stau = reinterpret_cast<T *>(b + FvpSmem<T>::st);
        T *sdt = stau + kFvEcap;
        uint4 *sa = reinterpret_cast<uint4 *>(b + FvpSmem<T>::sa);
        T *sg = reinterpret_cast<T *>(b + FvpSmem<T>::sg);
        const int nk = k + gridDim.x;
        FvItem nx;
        if (nk < nitem) {  // the next item's staging buffer, while this one computes
            nx = fv_item(W, nk);
            fvp_stage_buffer<T, STAGE>(smem_raw + (p ^ 1) * FvpSmem<T>::buf, nx, fin, tau, W, G, CG);
        }
        cp_async_commit();
        cp_async_wait_group<1>();  // everything of this item has landed (only the newest group may not)

        const int cnt = it.cnt, E = it.cnt + it.nh, NG = it.cnt + it.nr1;
        const InstParam *__restrict__ Pp = G.ip + G.tile_inst[it.base / kTile];
        const T rho0 = ipv<T>(Pp->rho0, Pp->rho0_f);
        const bool mine = t < cnt;
        const int i = it.base + t;
        if (STAGE == 1) {  // f^(1) of the cells this thread staged (their copies have landed)
            const T dtg = ipv<T>(Pp->dt, Pp->dt_f);
            for (int e = t; e < E; e += kFvThreads)
                fv_relax_row(sf, sf0, e, rho0, G.dtc != nullptr ? sdt[e] : dtg, stau[e]);
        }
        __syncthreads();

        // gradients and outgoing face values of item cells (geometry in their face-value rows)
        // and ring-1 cells (geometry in the staging buffer)
        T q[8];
        if (mine) {
            T lw[8];
            fv_load_vals(sv, t, 0, q);
            fv_load_vals(sv, t, 1, q + 4);
            fv_load_vals(sv, t, 2, lw);
            fv_load_vals(sv, t, 3, lw + 4);
            fv_cell<T>(t, q, lw, sa[t], sf, sf0[t], sv, G, rho0);
        }
        for (int c = (mine ? t + kFvThreads : t); c < NG; c += kFvThreads) {
            if (c < cnt) continue;
            T qr[8], lr[8];
            const T *g = sg + (c - cnt) * 16;   // swizzled like face-value row c
            const int cs = (c >> 1) & 3;
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
                qr[k4] = g[4 * (0 ^ cs) + k4];
                qr[4 + k4] = g[4 * (1 ^ cs) + k4];
                lr[k4] = g[4 * (2 ^ cs) + k4];
                lr[4 + k4] = g[4 * (3 ^ cs) + k4];
            }
            fv_cell<T>(c, qr, lr, sa[c], sf, sf0[c], sv, G, rho0);
        }
        __syncthreads();

        // the accumulator rows of this item (issued when the previous item finished)
        {
            long long itw = 0;
            bool done = W.wait_first > 0 ? mbar_try_wait(bar, phase) : mbar_test_wait(bar, phase);
            while (!done && ++itw < W.wait_first) done = mbar_try_wait(bar, phase);
            if (__syncthreads_or(!done)) {
                if (t == 0) atomicExch(W.err, 1);
                for (long long w = 0; w < kWaitLimit && !mbar_try_wait(bar, phase); ++w) {
                }
                cp_async_wait_all();  // nothing may land in shared memory after the CTA leaves
                return;
            }
        }

        double st[4] = {0.0, 0.0, 0.0, 0.0};
        if (mine) {
            T fi[kQ], acc[kQ];
            const uint4 wt = sa[t];
            V fr[4];
            fv_load_row(sf, t, fr);
            fi[0] = sf0[t];
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) {
                fi[fv_first(q2)] = fr[q2].x;
                fi[fv_second(q2)] = fr[q2].y;
            }
            fv_flux<T>(t, q, wt, fi, sv, G, rho0, acc);
            const InstParam P = *Pp;
            T macv[3];
            T uo = T(0), vo0 = T(0);
            if (STATS) {
                uo = mac[1 * np + i];
                vo0 = mac[2 * np + i];
            }
            const T tau_i = STAGE == 1 ? stau[t] : sacc[2 * kQ * kFvThreads + t];
            stage_algebra<T, STAGE, false, kFvThreads, false>(i, np, fi, acc, P, tau_i, cell_dt(G, P, i), sacc,
                                                              kFvThreads, t, sacc + kQ * kFvThreads, kFvThreads,
                                                              t, fs_out, fn, Bacc, Cacc, mac, nullptr, G.area,
                                                              nullptr, false, T(0), macv);
            if (STATS) {
                const double un = double(macv[1]), vn = double(macv[2]), r = double(macv[0]);
                const bool bad = !(isfinite(un) && isfinite(vn) && isfinite(r));
                st[0] = (un - double(uo)) * (un - double(uo)) + (vn - double(vo0)) * (vn - double(vo0));
                st[1] = un * un + vn * vn;
                st[2] = r * double(G.area[i]);
                st[3] = bad ? 1.0 : 0.0;
            }
        }
        if (STATS) block_sum<4, kFvThreads>(st, partial + 4 * k);
        __syncthreads();  // this item is done with the face values, the accumulators and its buffer
        if (nk < nitem) {
            fvp_stage_item_rows<T, STAGE>(nx, sv, sacc, bar, fin, Bacc, Cacc, tau, G, CG);
            cp_async_commit();  // its own group: the next iteration's wait covers it
            it = nx;
        }
    }
    cp_async_wait_all();
}
