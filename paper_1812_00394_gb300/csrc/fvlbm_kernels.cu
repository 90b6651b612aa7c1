// fvlbm_kernels.cu -- sm_103a kernels and the C ABI entry points of the FVLBM time step.
//
// One thread owns one cell.  Cells are Hilbert ordered per instance and instances are padded
// to a multiple of kBlock (two kTile tiles), so every thread block belongs to exactly one
// instance and reads that instance's parameters.  Every per-cell array is structure-of-arrays with stride
// np (all instances), so a warp reads 32 consecutive words per field.  Face fluxes are
// accumulated per cell over the cell's own face list (each interior face is evaluated by
// both of its cells with bit-identical face values), so no atomics are needed and the sum is
// deterministic.
//
// Step (Sec. 3.2, Steps 1-7) as launched per time step:
//   [k_sst_grad, k_sst_update]      Step 1 (k-omega SST, Eq. (SSTequint), Eq. (turbtau))
//   k_stage1                        stage 1: f^(1) from f^n (Eq. (fnewstage), J = 1)
//   k_grad, k_flux_stage<1>         Gamma^a(f^(1)) (Eq. (advection)); stage 2 solve
//   k_grad, k_flux_stage<2>         Gamma^a(f^(2)); stage 3 solve
//   k_grad, k_flux_stage<3>         Gamma^a(f^(3)); Eq. (imextwo); macros (Step 7)
// The stage algebra uses that the last row of the implicit tableau equals its weights:
//   f^{n+1} = f^(3) + dt (-1/6 Gamma^a(1) - 1/6 Gamma^a(2) + 1/3 Gamma^a(3)),
// and carries two accumulators B = f^n + dt/2 Gamma^a(1) + dt/3 (Gamma^c(1) + Gamma^c(2)) and
// C = -dt/6 (Gamma^a(1) + Gamma^a(2)) instead of all six Gamma arrays.
//
// Storage of f: the deviation f_alpha - w_alpha rho0, in double (FVLBM_FP64) or float
// (FVLBM_FP32_DEV).  Every map of the step is affine in f with weights summing to one, and
// the convection of a constant vanishes on closed cells, so the offset w_alpha rho0 drops out.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only; ranges cost a check unless a profiler is attached

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>
#include <vector>

#include "fvlbm_dual.h"
#include "fvlbm_internal.h"

namespace fvlbm {

// ------------------------------------------------------------------ lattice constants
__device__ __forceinline__ int ex_of(int a) {
    return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__device__ __forceinline__ int ey_of(int a) {
    return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
template <class T>
__device__ __forceinline__ T w_of(int a) {
    return a == 0 ? T(4.0 / 9.0) : (a < 5 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}
// e_alpha . (x, y) for a compile-time alpha (unrolled loops): the components are 0 or +-1, so
// the product is a sign change, a sum or a difference; writing it out keeps the compiler from
// issuing the multiplications by 0 that IEEE semantics would otherwise force.
template <class T>
__device__ __forceinline__ T edot(int a, T x, T y) {
    const int cx = ex_of(a), cy = ey_of(a);
    if (cx == 0 && cy == 0) return T(0);
    if (cx == 0) return cy > 0 ? y : -y;
    if (cy == 0) return cx > 0 ? x : -x;
    const T xs = cx > 0 ? x : -x;
    return cy > 0 ? xs + y : xs - y;
}

// SST constants (Sec. 2)
constexpr double kA1 = 0.31, kBstar = 0.09, kKappa = 0.41;
constexpr double kSk1 = 0.85, kSw1 = 0.5, kB1 = 0.075;
constexpr double kSk2 = 1.0, kSw2 = 0.856, kB2 = 0.0828;
constexpr double kCs2 = 1.0 / 3.0;

struct InstParam {
    double dt, nu, rho0, omega_min;
    int sst;      // 1: k-omega SST instance; 0: laminar (SST kernels skip its tiles)
    int local;    // 1: local time stepping (cell steps in Geo::dtc)
    int variant;  // reading variants: 1 limiter on grad f, 2 SST non-orthogonal correction,
                  // 4 SST per stage, 8 production limiter
    float dt_f, nu_f, rho0_f, omega_min_f;  // the same values rounded once, for float kernels
};

// An instance parameter in the kernel's type: float kernels read the pre-rounded copy instead
// of converting the double (a conversion that runs on the slow FP64 pipe of this GPU).
template <class T>
__device__ __forceinline__ T ipv(double d, float) {
    return T(d);
}
template <>
__device__ __forceinline__ float ipv<float>(double, float f) {
    return f;
}

constexpr int kXRow = kQ + 3;  // doubles per cell in a ghost-exchange row: f, k, omega, nu_t

template <class T>
struct Geo {
    const int *__restrict__ nbr;   // [4 np]
    const T *__restrict__ sn;      // [8 np]
    const T *__restrict__ lsq;     // [8 np]
    const T *__restrict__ rown;    // [8 np]
    const T *__restrict__ rnbr;    // [8 np]
    const T *__restrict__ dinv;    // [4 np]
    const T *__restrict__ area;    // [np]
    const T *__restrict__ wdist;   // [np]
    const int *__restrict__ tile_inst;
    const InstParam *__restrict__ ip;
    const int *__restrict__ btype;  // [nbt]
    const T *__restrict__ bval;     // [5 nbt] field-major: bval[c * nbt + b]
    const T *__restrict__ dtc;      // [np] local time step of each cell, or NULL (global dt)
    int np, nbt;
};

// Time step of cell i: its own under local time stepping, else the instance's.
template <class T>
__device__ __forceinline__ T cell_dt(const Geo<T> &G, const InstParam &P, int i) {
    return G.dtc != nullptr ? G.dtc[i] : ipv<T>(P.dt, P.dt_f);
}

// ------------------------------------------------------------------ cell algebra
// Quotient a / b in the collision and stage algebra and in the SST gradients (limiter, f1).
// In float it is the fast form (within 2 ulp instead of correctly rounded): the FP32 path
// stores deviations f - w rho0 whose rounding (~1e-9 of values ~1e-2) dominates it.  The SST
// update (point-implicit destruction, f2, nu_t) keeps correctly rounded division: measured on
// a 200k-cell airfoil after 1,000 steps, the FP32 velocity error against FP64 is 1.2e-5 either
// way for the stage algebra and the gradients, and 1.2e-4 with the fast form in the update.
template <class T>
__device__ __forceinline__ T sdiv(T a, T b) {
    if constexpr (std::is_same<T, float>::value)
        return __fdividef(a, b);
    else
        return a / b;
}

// Moments of a deviation vector d = f - w rho0: drho = sum d, rho = rho0 + drho, u = sum e d / rho.
template <class T>
__device__ __forceinline__ void moments(const T *d, T rho0, T &drho, T &rho, T &u, T &v) {
    T s = 0, jx = 0, jy = 0;
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        s += d[a];
        if (ex_of(a) > 0) jx += d[a];
        if (ex_of(a) < 0) jx -= d[a];
        if (ey_of(a) > 0) jy += d[a];
        if (ey_of(a) < 0) jy -= d[a];
    }
    drho = s;
    rho = rho0 + s;
    const T ir = sdiv(T(1), rho);
    u = jx * ir;
    v = jy * ir;
}

// Equilibrium deviation f^eq(rho, u) - w rho0 = w [drho + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)].
template <class T>
__device__ __forceinline__ void feq_dev(T drho, T rho, T u, T v, T *eq) {
    const T uu = T(1.5) * (u * u + v * v);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        const T eu = edot<T>(a, u, v);
        eq[a] = w_of<T>(a) * (drho + rho * (T(3) * eu + T(4.5) * eu * eu - uu));
    }
}

// Boundary face values f_{alpha,bc} (deviation form) from the owner cell: non-equilibrium
// extrapolation for wall / inlet / outlet, characteristic choice on the far field.
template <class T>
__device__ __forceinline__ void boundary_values(int type, const T *__restrict__ bval, int b,
                                                int nbt, T snx, T sny, const T *fP, T drP, T rP,
                                                T uP, T vP, T rho0, T *out) {
    T eqP[kQ], eqB[kQ];
    feq_dev(drP, rP, uP, vP, eqP);
    const T rb = bval[0 * nbt + b], ub = bval[1 * nbt + b], vb = bval[2 * nbt + b];
    if (type == FVLBM_BC_WALL || type == FVLBM_BC_INLET) {
        feq_dev(drP, rP, ub, vb, eqB);
#pragma unroll
        for (int a = 0; a < kQ; ++a) out[a] = eqB[a] + (fP[a] - eqP[a]);
    } else if (type == FVLBM_BC_OUTLET) {
        feq_dev(rb - rho0, rb, uP, vP, eqB);
#pragma unroll
        for (int a = 0; a < kQ; ++a) out[a] = eqB[a] + (fP[a] - eqP[a]);
    } else {
        feq_dev(rb - rho0, rb, ub, vb, eqB);
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            const T en = edot<T>(a, snx, sny);
            out[a] = en < T(0) ? eqB[a] : fP[a];
        }
    }
}

template <class T>
__device__ __forceinline__ void load9(const T *__restrict__ f, size_t np, int i, T *o) {
#pragma unroll
    for (int a = 0; a < kQ; ++a) o[a] = f[a * np + i];
}
template <class T>
__device__ __forceinline__ void store9(T *__restrict__ f, size_t np, int i, const T *o) {
#pragma unroll
    for (int a = 0; a < kQ; ++a) f[a * np + i] = o[a];
}

// ------------------------------------------------------------------ stage 1 (local)
// f^(1) = [f^n + (dt/tau)(1/4) f^eq(rho^n, u^n)] / (1 + (dt/tau)/4): Eq. (fnewstage), J = 1.
template <class T>
__device__ __forceinline__ void relax9(T *f, T rho0, T dt, T tau_i, T *eq_out = nullptr) {
    T eq[kQ], dr, r, u, v;
    moments(f, rho0, dr, r, u, v);
    feq_dev(dr, r, u, v, eq);
    const T zq = sdiv(dt, tau_i) * T(0.25);
    const T inv = sdiv(T(1), T(1) + zq);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        if (eq_out != nullptr) eq_out[a] = eq[a];  // f^eq(f^n), for a later stage-1 algebra
        f[a] = (f[a] + zq * eq[a]) * inv;
    }
}

template <class T>
__global__ void __launch_bounds__(kTile) k_stage1(const T *__restrict__ fn, T *__restrict__ fs,
                                                  const T *__restrict__ tau, Geo<T> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    T f[kQ];
    load9(fn, np, i, f);
    relax9(f, ipv<T>(P.rho0, P.rho0_f), cell_dt(G, P, i), tau[i]);
    store9(fs, np, i, f);
}

// Macros (rho, u, v) of a stage value, for the SST solve before the next stage (per-stage
// SST reading).
template <class T>
__global__ void __launch_bounds__(kTile) k_stage_macros(const T *__restrict__ fs, T *__restrict__ mac,
                                                        Geo<T> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    T f[kQ], dr, r, u, v;
    load9(fs, np, i, f);
    const InstParam &P = G.ip[G.tile_inst[blockIdx.x]];
    moments(f, ipv<T>(P.rho0, P.rho0_f), dr, r, u, v);
    mac[i] = r;
    mac[np + i] = u;
    mac[2 * np + i] = v;
}

// ------------------------------------------------------------------ gradient of f
// Least-squares cell gradient (Step 2): g_i = sum_m W_m (f_m - f_i), data from face neighbours
// and, on boundary faces, the boundary value at the face midpoint.
template <class T, bool LIMIT>
__global__ void __launch_bounds__(kTile) k_grad(const T *__restrict__ f, T *__restrict__ g,
                                                Geo<T> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    const T rho0 = ipv<T>(P.rho0, P.rho0_f);
    T fi[kQ], gx[kQ], gy[kQ], lo[kQ], hi[kQ];
    load9(f, np, i, fi);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        gx[a] = gy[a] = T(0);
        lo[a] = hi[a] = fi[a];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + i];
        if (nb == kNone) continue;
        const T wx = G.lsq[(2 * m) * np + i], wy = G.lsq[(2 * m + 1) * np + i];
        if (nb >= 0) {
#pragma unroll
            for (int a = 0; a < kQ; ++a) {
                const T fm = f[a * np + nb];
                const T d = fm - fi[a];
                gx[a] += wx * d;
                gy[a] += wy * d;
                if (LIMIT) {
                    lo[a] = fmin(lo[a], fm);
                    hi[a] = fmax(hi[a], fm);
                }
            }
        } else {
            const int b = -nb - 1;
            T dr, r, u, v, fb[kQ];
            moments(fi, rho0, dr, r, u, v);
            boundary_values(G.btype[b], G.bval + b, 0, G.nbt, G.sn[(2 * m) * np + i],
                            G.sn[(2 * m + 1) * np + i], fi, dr, r, u, v, rho0, fb);
#pragma unroll
            for (int a = 0; a < kQ; ++a) {
                const T d = fb[a] - fi[a];
                gx[a] += wx * d;
                gy[a] += wy * d;
                if (LIMIT) {
                    lo[a] = fmin(lo[a], fb[a]);
                    hi[a] = fmax(hi[a], fb[a]);
                }
            }
        }
    }
    if (LIMIT && (P.variant & 1)) {
        // Venkatakrishnan limiter (reading variant 1): phi = min over faces of
        // [(D1^2 + e2) D2 + 2 D2^2 D1] / [D1^2 + 2 D2^2 + D1 D2 + e2] / D2, D2 = g . r_m the
        // increment to face m, D1 the distance to the max (D2 > 0) or min (D2 < 0) of the cell
        // and its face data, e2 = A^(3/2).
        const T ar = G.area[i];
        const T e2 = ar * sqrt(ar);
        T phi[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) phi[a] = T(1);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (G.nbr[m * np + i] == kNone) continue;
            const T rx = G.rown[(2 * m) * np + i], ry = G.rown[(2 * m + 1) * np + i];
#pragma unroll
            for (int a = 1; a < kQ; ++a) {
                const T d2 = gx[a] * rx + gy[a] * ry;
                if (d2 == T(0)) continue;
                const T d1 = d2 > T(0) ? hi[a] - fi[a] : lo[a] - fi[a];
                const T r = ((d1 * d1 + e2) * d2 + T(2) * d2 * d2 * d1) /
                            (d1 * d1 + T(2) * d2 * d2 + d1 * d2 + e2) / d2;
                phi[a] = fmin(phi[a], r);
            }
        }
#pragma unroll
        for (int a = 1; a < kQ; ++a) {
            gx[a] *= phi[a];
            gy[a] *= phi[a];
        }
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        g[(2 * a) * np + i] = gx[a];
        g[(2 * a + 1) * np + i] = gy[a];
    }
}

// ------------------------------------------------------------------ block reduction (FP64)
template <int N, int NT = kTile>
__device__ __forceinline__ void block_sum(double (&v)[N], double *out) {
    __shared__ double red[NT / 32][N];
#pragma unroll
    for (int k = 0; k < N; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < N; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < N) {
        double s = 0;
        for (int w = 0; w < NT / 32; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Local algebra after Gamma^a(J) of a cell is known (acc = -Gamma^a(J)); fi = f^(J).
//   J = 1: Gamma^c(1) from f^n and f^(1); stage 2 solve (Eq. (fnewstage)); B, C
//   J = 2: stage 3 solve from B + dt/2 Gamma^a(2); C update
//   J = 3: f^{n+1} = f^(3) + C + dt/3 Gamma^a(3) (Eq. (imextwo)); macros; FP64 partial sums
//   J = 4: explicit Euler comparison scheme, f^{n+1} = f^n + dt (Gamma^a + Gamma^c), into fs_out
// The accumulator inputs are read through (pointer, row stride, column): a1 is f^n (J = 1),
// B (J = 2) or C (J = 3); a2 is C (J = 2).  Outputs go to global memory at cell i.
//   FN_FROM_F1: unless fn_read, f^n is not read but recovered from f^(1) = [f^n + z/4 f^eq] /
//   (1 + z/4) as f^n = f^(1) - dt/4 Gamma^c(1) (same moments, so f^eq(1) follows from f^(1));
//   the recovery multiplies the rounding of f^(1) by z/4, so with large z (local time steps)
//   the caller sets fn_read and f^n is read from fn at cell i instead;
//   frel (if given): at J = 3, laminar instances also store f^(1) of the next step.
// The collision terms are formed from differences that are not scaled by z: with
// f^(J) = (X + zJ f^eq) / (1 + zJ), dt Gamma^c(J) = dt/tau (f^eq - X) / (1 + zJ) exactly, so a
// rounding of X or f^eq is multiplied by dt/tau / (1 + zJ) <= 1/m_JJ instead of dt/tau.
// Store of a stage value f^(2) or f^(3): structure of arrays, or (ROWS) the cell-major rows of
// the face-value stages: alpha = 1..8 in pair order (1,3)(2,4)(5,7)(6,8) at f[8 i] (the two
// halves swapped where bit 2 of i is set), f_0 at f[8 np + i].
template <class T, bool ROWS>
__device__ __forceinline__ void store_stage(T *__restrict__ f, size_t np, int i, const T *o) {
    if constexpr (!ROWS) {
        store9(f, np, i, o);
    } else {
        T *row = f + 8 * static_cast<size_t>(i);
        const int sw = (i & 4) ? 4 : 0;  // halves swapped where bit 2 of the cell index is set
        if constexpr (std::is_same<T, float>::value) {
            *reinterpret_cast<float4 *>(row + sw) = make_float4(o[1], o[3], o[2], o[4]);
            *reinterpret_cast<float4 *>(row + (sw ^ 4)) = make_float4(o[5], o[7], o[6], o[8]);
        } else {
            *reinterpret_cast<double2 *>(row + sw) = make_double2(o[1], o[3]);
            *reinterpret_cast<double2 *>(row + sw + 2) = make_double2(o[2], o[4]);
            *reinterpret_cast<double2 *>(row + (sw ^ 4)) = make_double2(o[5], o[7]);
            *reinterpret_cast<double2 *>(row + (sw ^ 4) + 2) = make_double2(o[6], o[8]);
        }
        f[8 * np + i] = o[0];
    }
}

// EQ1_IN_A2 (stage 1): f^eq(f^n) is given in a2 (the face-value stage relaxed the cell with it).
template <class T, int STAGE, bool STATS, int NT, bool FN_FROM_F1 = false, bool ROWS = false,
          bool EQ1_IN_A2 = false>
__device__ __forceinline__ void stage_algebra(int i, size_t np, const T *fi, const T *acc,
                                              const InstParam &P, T t_i, T dt_i, const T *a1, size_t ld1,
                                              int c1, const T *a2, size_t ld2, int c2,
                                              T *__restrict__ fs_out, T *__restrict__ fn,
                                              T *__restrict__ Bacc, T *__restrict__ Cacc,
                                              T *__restrict__ mac, double *__restrict__ partial,
                                              const T *__restrict__ area,
                                              T *__restrict__ frel = nullptr,
                                              bool fn_read = false, T t1_i = T(0),
                                              T *macv = nullptr) {
    const T rho0 = ipv<T>(P.rho0, P.rho0_f);
    const T dt = dt_i;
    const T itau = sdiv(T(1), t_i);     // one division per cell, products below
    const T dt3 = dt * T(1.0 / 3.0), dt6 = dt * T(1.0 / 6.0);
    if (STAGE == 1) {
        // fi = f^(1); f^n and dt Gamma^c(1)
        T f0[kQ], eq[kQ], X[kQ], dr, r, u, v;
        T dgc1[kQ];
        const T z = dt * itau;
        const T zq = z * T(0.25);
        const T inv = sdiv(T(1), T(1) + zq);
        if (FN_FROM_F1 && !fn_read) {
            moments(fi, rho0, dr, r, u, v);
            feq_dev(dr, r, u, v, eq);
#pragma unroll
            for (int a = 0; a < kQ; ++a) {
                dgc1[a] = (eq[a] - fi[a]) * z;
                f0[a] = fi[a] - T(0.25) * dgc1[a];
            }
        } else {
#pragma unroll
            for (int a = 0; a < kQ; ++a) f0[a] = FN_FROM_F1 ? fn[a * np + i] : a1[a * ld1 + c1];
            if constexpr (EQ1_IN_A2) {
#pragma unroll
                for (int a = 0; a < kQ; ++a) eq[a] = a2[a * ld2 + c2];
            } else {
                moments(f0, rho0, dr, r, u, v);
                feq_dev(dr, r, u, v, eq);
            }
            // f^(1) = (f^n + zq1 f^eq) / (1 + zq1), relaxed with tau^(1) (= tau unless the SST
            // is solved per stage, when stage 2 has its own tau)
            T s1 = z * inv;
            if (t1_i > T(0)) {
                const T z1 = sdiv(dt, t1_i);
                s1 = sdiv(z1, T(1) + T(0.25) * z1);
            }
#pragma unroll
            for (int a = 0; a < kQ; ++a) dgc1[a] = (eq[a] - f0[a]) * s1;
        }
#pragma unroll
        for (int a = 0; a < kQ; ++a) X[a] = f0[a] - T(0.5) * dt * acc[a];
        moments(X, rho0, dr, r, u, v);
        feq_dev(dr, r, u, v, eq);
        const T s2 = z * inv;
        T f2[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            f2[a] = (X[a] + zq * eq[a]) * inv;
            const T dgc2 = (eq[a] - X[a]) * s2;  // dt Gamma^c(2)
            Bacc[a * np + i] = X[a] + T(1.0 / 3.0) * (dgc1[a] + dgc2);
            Cacc[a * np + i] = dt6 * acc[a];
        }
        store_stage<T, ROWS>(fs_out, np, i, f2);
    } else if (STAGE == 2) {
        T X[kQ], eq[kQ], dr, r, u, v, f3[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) X[a] = a1[a * ld1 + c1] - T(0.5) * dt * acc[a];
        moments(X, rho0, dr, r, u, v);
        feq_dev(dr, r, u, v, eq);
        const T zt = dt3 * itau;
        const T inv = sdiv(T(1), T(1) + zt);
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            f3[a] = (X[a] + zt * eq[a]) * inv;
            Cacc[a * np + i] = a2[a * ld2 + c2] + dt6 * acc[a];
        }
        store_stage<T, ROWS>(fs_out, np, i, f3);
    } else if (STAGE == 4) {
        // explicit Euler (comparison scheme): f^{n+1} = f^n + dt [Gamma^a + Gamma^c](f^n)
        T eq[kQ], fnew[kQ], dr, r, u, v;
        moments(fi, rho0, dr, r, u, v);
        feq_dev(dr, r, u, v, eq);
#pragma unroll
        for (int a = 0; a < kQ; ++a) fnew[a] = fi[a] + dt * (-acc[a] + (eq[a] - fi[a]) * itau);
        store9(fs_out, np, i, fnew);
        moments(fnew, rho0, dr, r, u, v);
        if (STATS) {
            const double uo = double(mac[1 * np + i]), vo = double(mac[2 * np + i]);
            const double un = double(u), vn = double(v);
            const bool bad = !(isfinite(un) && isfinite(vn) && isfinite(double(r)));
            double s[4] = {(un - uo) * (un - uo) + (vn - vo) * (vn - vo), un * un + vn * vn,
                           double(r) * double(area[i]), bad ? 1.0 : 0.0};
            block_sum<4, NT>(s, partial + 4 * blockIdx.x);
        }
        mac[0 * np + i] = r;
        mac[1 * np + i] = u;
        mac[2 * np + i] = v;
    } else {
        T fnew[kQ], dr, r, u, v;
#pragma unroll
        for (int a = 0; a < kQ; ++a) fnew[a] = fi[a] + a1[a * ld1 + c1] - dt3 * acc[a];
        store9(fn, np, i, fnew);
        moments(fnew, rho0, dr, r, u, v);
        if (STATS) {
            const double uo = double(mac[1 * np + i]), vo = double(mac[2 * np + i]);
            const double un = double(u), vn = double(v);
            const bool bad = !(isfinite(un) && isfinite(vn) && isfinite(double(r)));
            double s[4] = {(un - uo) * (un - uo) + (vn - vo) * (vn - vo), un * un + vn * vn,
                           double(r) * double(area[i]), bad ? 1.0 : 0.0};
            block_sum<4, NT>(s, partial + 4 * blockIdx.x);
        }
        mac[0 * np + i] = r;
        mac[1 * np + i] = u;
        mac[2 * np + i] = v;
        if (macv) {  // the new macros, for a caller that forms the statistics itself
            macv[0] = r;
            macv[1] = u;
            macv[2] = v;
        }
        if (frel != nullptr && !P.sst) {  // laminar: tau is constant, relax for the next step
            relax9(fnew, rho0, dt, t_i);
            store9(frel, np, i, fnew);
        }
    }
}

// Stage algebra with accumulators in global memory (two-pass kernels).
template <class T, int STAGE, bool STATS, int NT>
__device__ __forceinline__ void stage_update(int i, size_t np, const T *fi, const T *acc,
                                             const InstParam &P, T *__restrict__ fs_out,
                                             T *__restrict__ fn, T *__restrict__ Bacc,
                                             T *__restrict__ Cacc, const T *__restrict__ tau,
                                             T *__restrict__ mac, double *__restrict__ partial,
                                             const T *__restrict__ area, T dt_i, T t1_i) {
    const T *a1 = STAGE == 1 ? fn : (STAGE == 2 ? Bacc : Cacc);
    stage_algebra<T, STAGE, STATS, NT>(i, np, fi, acc, P, tau[i], dt_i, a1, np, i, Cacc, np, i, fs_out,
                                       fn, Bacc, Cacc, mac, partial, area, nullptr, false, t1_i);
}

// ------------------------------------------------------------------ flux + stage solve
// Gamma^a_alpha,i = -sum_m (e_alpha . n_m Delta l_m / A_i) f_{alpha,bc,m}  (Eq. (advection)) with
// upwind linear face values, then the local algebra of the next stage (see file header).
template <class T, int STAGE, bool STATS>
__global__ void __launch_bounds__(kTile)
    k_flux_stage(const T *__restrict__ fs, const T *__restrict__ g, T *__restrict__ fs_out,
                 T *__restrict__ fn, T *__restrict__ Bacc, T *__restrict__ Cacc,
                 const T *__restrict__ tau, T *__restrict__ mac, double *__restrict__ partial,
                 Geo<T> G, const T *__restrict__ tau1 = nullptr) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    const T rho0 = ipv<T>(P.rho0, P.rho0_f);
    T fi[kQ], acc[kQ];
    load9(fs, np, i, fi);
#pragma unroll
    for (int a = 0; a < kQ; ++a) acc[a] = T(0);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + i];
        if (nb == kNone) continue;
        const T snx = G.sn[(2 * m) * np + i], sny = G.sn[(2 * m + 1) * np + i];
        if (nb >= 0) {
            const T rox = G.rown[(2 * m) * np + i], roy = G.rown[(2 * m + 1) * np + i];
            const T rnx = G.rnbr[(2 * m) * np + i], rny = G.rnbr[(2 * m + 1) * np + i];
#pragma unroll
            for (int a = 0; a < kQ; ++a) {
                const T en = edot<T>(a, snx, sny);
                T fv;
                if (en >= T(0))
                    fv = fi[a] + g[(2 * a) * np + i] * rox + g[(2 * a + 1) * np + i] * roy;
                else
                    fv = fs[a * np + nb] + g[(2 * a) * np + nb] * rnx + g[(2 * a + 1) * np + nb] * rny;
                acc[a] += en * fv;
            }
        } else {
            const int b = -nb - 1;
            T dr, r, u, v, fb[kQ];
            moments(fi, rho0, dr, r, u, v);
            boundary_values(G.btype[b], G.bval + b, 0, G.nbt, snx, sny, fi, dr, r, u, v, rho0, fb);
#pragma unroll
            for (int a = 0; a < kQ; ++a) acc[a] += edot<T>(a, snx, sny) * fb[a];
        }
    }
    stage_update<T, STAGE, STATS, kTile>(i, np, fi, acc, P, fs_out, fn, Bacc, Cacc, tau, mac, partial,
                                         G.area, cell_dt(G, P, i),
                                         (STAGE == 1 && tau1 != nullptr) ? tau1[i] : T(0));
}

// ------------------------------------------------------------------ fused stage kernel
// Per block of kBlock consecutive cells (compact patch, see the host renumbering): the ring-1
// and ring-2 halo cells are listed on the host; the local adjacency of block and ring-1 cells
// is stored with 16-bit local indices.  Encoding of one adjacency word: kAdjNone (no face),
// kAdjBnd | global boundary face, or local index | back slot << 16 | (neighbour is a
// triangle) << 18.
constexpr int kFusedSmemCap = 200 * 1024;  // dynamic shared memory cap of the fused kernel
constexpr unsigned kAdjNone = 0xFFFFFFFFu;
constexpr unsigned kAdjBnd = 0x80000000u;
constexpr long long kWaitLimit = 1ll << 26;  // bounded spin on the staging barrier

struct Halo {
    const int *__restrict__ halo_ptr;   // [nblk + 1] offsets into halo
    const int *__restrict__ halo;       // global ids: ring 1 then ring 2, per block
    const int *__restrict__ r1;         // [nblk] ring-1 count
    const int *__restrict__ adj_ptr;    // [nblk + 1] offsets (cells) into adj / 4
    const unsigned *__restrict__ adj;   // per block [4][kBlock + r1] adjacency words
    int *__restrict__ err;              // set to 1 if a staging wait gave up
    int emax, gmax;                     // smem row strides: max ext cells, max gradient cells
    long long wait_first;               // polls of the first staging wait (fvlbm_set_wait_limit)
};

// Compact geometry of the fused kernels: per cell the node positions relative to the centroid
// (gq, face m joins nodes m and m+1) and, per face slot, d_m = neighbour centroid (periodic
// shift included) or face midpoint, minus the own centroid.  Everything else is derived:
// area and n dl / A from gq, the face offset r_m = face midpoint - centroid from gq, the
// neighbour's offset r_m - d_m, and the least-squares weights M^{-1} d_m.
template <class T>
struct CompactGeo {
    const T *__restrict__ gq;    // [8 np]
    const T *__restrict__ dv;    // [8 np]
};

// ---- asynchronous staging primitives (sm_90+ bulk copy engine and cp.async)
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count = 1) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Loads of small tables that every launch reads once per item (the face-value items' headers
// and halo ids), marked evict-last in L2 so that the streamed state does not push them out
// between launches: their load is the first memory round trip of every CTA.
__device__ __forceinline__ unsigned long long l2_keep_policy() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int ld_keep(const int *a, unsigned long long pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_keep(const float *a, unsigned long long pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_keep(const double *a, unsigned long long pol) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ int4 ld_keep(const int4 *a, unsigned long long pol) {
    int4 v;
    asm("ld.global.nc.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(a), "l"(pol));
    return v;
}

// Face m of a cell whose node positions (relative to its centroid) are q[(2k + c) * ld]:
// midpoint r = (q_m + q_{m+1}) / 2 and edge vector e = q_{m+1} - q_m.
template <class T>
__device__ __forceinline__ void face_geo_s(const T *q, int ld, int m, int nv, T &rx, T &ry,
                                           T &exv, T &eyv) {
    const int m1 = (m + 1 == nv) ? 0 : m + 1;
    const T x0 = q[(2 * m) * ld], y0 = q[(2 * m + 1) * ld];
    const T x1 = q[(2 * m1) * ld], y1 = q[(2 * m1 + 1) * ld];
    rx = T(0.5) * (x0 + x1);
    ry = T(0.5) * (y0 + y1);
    exv = x1 - x0;
    eyv = y1 - y0;
}

// Shared-memory layout of the fused kernel (element offsets, every row 16-byte aligned):
//   sf  [9][emax]   f^(J) of block, ring-1 and ring-2 cells
//   sg  [gmax][17]  gradients (alpha = 1..8; x, y) of block and ring-1 cells, cell-major
//   sD  [8][gmax]   neighbour-centroid offsets d_m of block and ring-1 cells
//   adj [4 gmax] words, then one 8-byte mbarrier

// Gradients in shared memory are cell-major, 16 values (alpha = 1..8, x and y) in a row of 17
// words: one base address per cell serves all 16 reads (immediate offsets), and the odd row
// length keeps consecutive cells in distinct banks.
constexpr int kGradStride = 17;

template <class T>
struct FusedSmem {
    static __host__ __device__ size_t elems(int emax, int gmax) {
        return size_t(kQ) * emax + size_t(kGradStride) * gmax + 8u * gmax;
    }
    static __host__ __device__ size_t bytes(int emax, int gmax) {
        return elems(emax, gmax) * sizeof(T) + 4u * gmax * sizeof(unsigned) + 16;
    }
};

// One IMEX stage for a block of BLK cells (BLK = 128 or 256), one thread per cell.  Staging: the block's own
// rows (contiguous in every SoA array) arrive by bulk copies on one mbarrier; halo rows are
// gathered with cp.async; each thread's accumulators, tau and face normals go straight into
// registers; nothing is waited for until everything has been issued.  Then: least-squares
// gradients of block + ring-1 cells, and per block cell the flux of Eq. (advection) and the
// local stage algebra.  No gradient array goes through HBM.  alpha = 0 has e = 0: no gradient
// and no flux.  Stage 1 stages f^(1), which the previous step (laminar instances) or the SST
// update (turbulent instances, with the new tau) has already relaxed from f^n; stage 3 writes
// f^(1) of the next step for laminar instances into frel.
template <class T, int STAGE, bool STATS, int BLK>
__global__ void __launch_bounds__(BLK, sizeof(T) == 4 ? (768 / BLK) : 1)
    k_fused_stage(const T *__restrict__ fin, T *__restrict__ fs_out, T *__restrict__ fn,
                  T *__restrict__ Bacc, T *__restrict__ Cacc, const T *__restrict__ tau,
                  T *__restrict__ mac, double *__restrict__ partial, Geo<T> G, Halo H,
                  T *__restrict__ frel, CompactGeo<T> CG) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int E0 = H.emax, G0 = H.gmax;
    T *sf = reinterpret_cast<T *>(smem_raw);
    T *sg = sf + kQ * E0;
    T *sD = sg + kGradStride * G0;
    unsigned *sAdj = reinterpret_cast<unsigned *>(sD + 8 * G0);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(sAdj + 4 * G0);

    const int b = blockIdx.x, t = threadIdx.x;
    const int base = b * BLK;
    const int i = base + t;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[b * (BLK / kTile)]];
    const T rho0 = ipv<T>(P.rho0, P.rho0_f);
    const int h0 = H.halo_ptr[b], nh = H.halo_ptr[b + 1] - h0, nr1 = H.r1[b];
    const int E = BLK + nh, NG = BLK + nr1;
    const unsigned *__restrict__ adj_g = H.adj + 4 * static_cast<size_t>(H.adj_ptr[b]);

    // 1. issue every copy of the block's data, then wait once
    if (t == 0) mbar_init(bar);
    __syncthreads();
    if (t == 0) {
        constexpr unsigned row = BLK * sizeof(T);
        const unsigned adj_bytes = 4u * NG * sizeof(unsigned);
        mbar_expect_tx(bar, row * (kQ + 8) + adj_bytes);
        for (int a = 0; a < kQ; ++a) bulk_g2s(sf + a * E0, fin + a * np + base, row, bar);
        for (int k = 0; k < 8; ++k) bulk_g2s(sD + k * G0, CG.dv + k * np + base, row, bar);
        bulk_g2s(sAdj, adj_g, adj_bytes, bar);
    }
    for (int e = BLK + t; e < E; e += BLK) {  // halo rows
        const int gid = H.halo[h0 + e - BLK];
#pragma unroll
        for (int a = 0; a < kQ; ++a) cp_async<sizeof(T)>(sf + a * E0 + e, fin + a * np + gid);
        if (e < NG) {
#pragma unroll
            for (int k = 0; k < 8; ++k) cp_async<sizeof(T)>(sD + k * G0 + e, CG.dv + k * np + gid);
        }
    }
    // this thread's accumulators, tau and node positions, straight into registers
    T a1[kQ], a2[kQ], q[8];
    const T tau_i = tau[i];
    {
        if (STAGE != 1) {
            const T *p1 = STAGE == 2 ? Bacc : Cacc;
#pragma unroll
            for (int a = 0; a < kQ; ++a) a1[a] = p1[a * np + i];
        }
        if (STAGE == 2) {
#pragma unroll
            for (int a = 0; a < kQ; ++a) a2[a] = Cacc[a * np + i];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = CG.gq[k * np + i];
    }
    cp_async_wait_all();
    {
        long long it = 0;
        // (a limit of 0 gives up at once, without polling: the diagnostic of the error path)
        bool done = H.wait_first > 0 && mbar_try_wait(bar, 0);
        while (!done && ++it < H.wait_first) done = mbar_try_wait(bar, 0);
        // the block leaves together if any thread gave up: flag it, wait once more (bounded)
        if (__syncthreads_or(!done)) {
            if (t == 0) atomicExch(H.err, 1);
            for (long long k = 0; k < kWaitLimit && !mbar_try_wait(bar, 0); ++k) {
            }
            return;
        }
    }

    // 2. least-squares gradients (alpha = 1..8) of block and ring-1 cells (Step 2)
    for (int c = t; c < NG; c += BLK) {
        T fc[kQ], gx[kQ], gy[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            fc[a] = sf[a * E0 + c];
            gx[a] = gy[a] = T(0);
        }
        // least-squares matrix M = sum_m d_m d_m^T of this cell, inverted once
        T mxx = 0, mxy = 0, myy = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (sAdj[m * NG + c] == kAdjNone) continue;
            const T dx = sD[(2 * m) * G0 + c], dy = sD[(2 * m + 1) * G0 + c];
            mxx += dx * dx;
            mxy += dx * dy;
            myy += dy * dy;
        }
        const T idet = T(1) / (mxx * myy - mxy * mxy);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const unsigned w = sAdj[m * NG + c];
            if (w == kAdjNone) continue;
            const T dx = sD[(2 * m) * G0 + c], dy = sD[(2 * m + 1) * G0 + c];
            const T wx = (myy * dx - mxy * dy) * idet, wy = (mxx * dy - mxy * dx) * idet;
            if (w & kAdjBnd) {
                const int bf = static_cast<int>(w & ~kAdjBnd);
                // outward face normal (n dl / A) for the far-field upwind choice
                const int gid = c < BLK ? base + c : H.halo[h0 + c - BLK];
                const T nx = G.sn[(2 * m) * np + gid], ny = G.sn[(2 * m + 1) * np + gid];
                T dr, r, u, v, fb[kQ];
                moments(fc, rho0, dr, r, u, v);
                boundary_values(G.btype[bf], G.bval + bf, 0, G.nbt, nx, ny, fc, dr, r, u, v, rho0,
                                fb);
#pragma unroll
                for (int a = 1; a < kQ; ++a) {
                    const T d = fb[a] - fc[a];
                    gx[a] += wx * d;
                    gy[a] += wy * d;
                }
            } else {
                const int j = static_cast<int>(w & 0xFFFFu);
#pragma unroll
                for (int a = 1; a < kQ; ++a) {
                    const T d = sf[a * E0 + j] - fc[a];
                    gx[a] += wx * d;
                    gy[a] += wy * d;
                }
            }
        }
#pragma unroll
        for (int a = 1; a < kQ; ++a) {
            sg[c * kGradStride + 2 * a - 2] = gx[a];
            sg[c * kGradStride + 2 * a - 1] = gy[a];
        }
    }
    __syncthreads();

    // 3. flux of block cell t (Eq. (advection)), then the stage algebra
    T fi[kQ], acc[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        fi[a] = sf[a * E0 + t];
        acc[a] = T(0);
    }
    const bool tri = sAdj[3 * NG + t] == kAdjNone;
    // end node of face m (m compile-time): node m + 1, wrapping to node 0 after the last face
    auto end_x = [&](int m) { return m == 3 ? q[0] : (m == 2 && tri ? q[0] : q[2 * m + 2]); };
    auto end_y = [&](int m) { return m == 3 ? q[1] : (m == 2 && tri ? q[1] : q[2 * m + 3]); };
    T a2x = T(0);  // twice the area (shoelace on centroid-relative nodes)
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (m < 3 || !tri) a2x += q[2 * m] * end_y(m) - end_x(m) * q[2 * m + 1];
    const T inv_a = a2x > T(0) ? sdiv(T(2), a2x) : T(0);  // padding cells have no faces
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const unsigned w = sAdj[m * NG + t];
        if (w == kAdjNone) continue;
        const T x1 = end_x(m), y1 = end_y(m);
        const T snx = (y1 - q[2 * m + 1]) * inv_a;   // n dl / A
        const T sny = -(x1 - q[2 * m]) * inv_a;
        if (w & kAdjBnd) {
            const int bf = static_cast<int>(w & ~kAdjBnd);
            T dr, r, u, v, fb[kQ];
            moments(fi, rho0, dr, r, u, v);
            boundary_values(G.btype[bf], G.bval + bf, 0, G.nbt, snx, sny, fi, dr, r, u, v, rho0, fb);
#pragma unroll
            for (int a = 1; a < kQ; ++a) acc[a] += edot<T>(a, snx, sny) * fb[a];
        } else {
            const int j = static_cast<int>(w & 0xFFFFu);
            // face offsets from this cell's centroid and from the neighbour's
            const T rox = T(0.5) * (q[2 * m] + x1), roy = T(0.5) * (q[2 * m + 1] + y1);
            const T rnx = rox - sD[(2 * m) * G0 + t], rny = roy - sD[(2 * m + 1) * G0 + t];
#pragma unroll
            for (int a = 1; a < kQ; ++a) {
                const T en = edot<T>(a, snx, sny);
                const bool own = en >= T(0);           // upwind side, branch free
                const int src = own ? t : j;
                const T rx = own ? rox : rnx, ry = own ? roy : rny;
                const T *gs = sg + src * kGradStride;
                const T fv = sf[a * E0 + src] + gs[2 * a - 2] * rx + gs[2 * a - 1] * ry;
                acc[a] += en * fv;
            }
        }
    }
    stage_algebra<T, STAGE, STATS, BLK, true>(i, np, fi, acc, P, tau_i, cell_dt(G, P, i), a1, 1, 0, a2, 1,
                                                        0, fs_out, fn, Bacc, Cacc, mac, partial,
                                                        G.area, frel, P.local != 0);  // local steps: read f^n
}

// Sum per-block partials into per-instance totals (one block per instance).
__global__ void k_reduce_instances(const double *__restrict__ partial,
                                   const int *__restrict__ inst_tile0, double *__restrict__ out) {
    const int inst = blockIdx.x;
    const int t0 = inst_tile0[inst], t1 = inst_tile0[inst + 1];
    double s[4] = {0, 0, 0, 0};
    for (int t = t0 + threadIdx.x; t < t1; t += kTile)
        for (int k = 0; k < 4; ++k) s[k] += partial[4 * t + k];
    block_sum<4>(s, out + 4 * inst);
}

#include "fvlbm_fused_fv.cuh"

// ------------------------------------------------------------------ SST (Step 1)
// ---- per-cell SST arithmetic, shared by the two-pass and the fused kernels
// Boundary values of (u, v, k, omega) on boundary face b of a cell with values (ui, vi, ki, wi)
// and wall distance di (Menter 1994 boundary conditions; wall omega = 60 nu / (beta1 d^2)).
template <class T>
__device__ __forceinline__ void sst_bvals(const Geo<T> &G, int b, T nu, T ui, T vi, T ki, T wi,
                                          T di, T &ub, T &vb, T &kb, T &wb) {
    const int t = G.btype[b];
    if (t == FVLBM_BC_WALL) {
        ub = G.bval[1 * G.nbt + b]; vb = G.bval[2 * G.nbt + b]; kb = T(0);
        wb = T(60) * nu / (T(kB1) * di * di);
    } else if (t == FVLBM_BC_OUTLET) {
        ub = ui; vb = vi; kb = ki; wb = wi;
    } else {
        ub = G.bval[1 * G.nbt + b]; vb = G.bval[2 * G.nbt + b];
        kb = G.bval[3 * G.nbt + b]; wb = G.bval[4 * G.nbt + b];
    }
}

// Gradients of u, v, k, omega (least squares; face data q[m] = neighbour or boundary values,
// has[m] = face present), Barth-Jespersen limited k / omega gradients for the upwind face
// values, and the blending function f1 = tanh(arg1^4) (Sec. 2, kinematic form).
template <class T>
__device__ __forceinline__ void sst_cell_grad(T ki, T wi, T di, T nu, const bool *has,
                                              const T (*q)[4], const T *W, const T *R,
                                              const T *uvkw_i, T *g, T *lg, T &f1) {
#pragma unroll
    for (int c = 0; c < 8; ++c) g[c] = T(0);
    T kq[4], wq[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        kq[m] = ki;
        wq[m] = wi;
        if (!has[m]) continue;
        const T du = q[m][0] - uvkw_i[0], dv = q[m][1] - uvkw_i[1];
        const T dk = q[m][2] - ki, dw = q[m][3] - wi;
        kq[m] = ki + dk;
        wq[m] = wi + dw;
        const T wx = W[2 * m], wy = W[2 * m + 1];
        g[0] += wx * du; g[1] += wy * du;
        g[2] += wx * dv; g[3] += wy * dv;
        g[4] += wx * dk; g[5] += wy * dk;
        g[6] += wx * dw; g[7] += wy * dw;
    }
    T klo = ki, khi = ki, wlo = wi, whi = wi;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        klo = fmin(klo, kq[m]); khi = fmax(khi, kq[m]);
        wlo = fmin(wlo, wq[m]); whi = fmax(whi, wq[m]);
    }
    T pk = T(1), pw = T(1);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (!has[m]) continue;
        const T rx = R[2 * m], ry = R[2 * m + 1];
        const T dkf = g[4] * rx + g[5] * ry, dwf = g[6] * rx + g[7] * ry;
        if (dkf > T(0)) pk = fmin(pk, sdiv(khi - ki, dkf));
        else if (dkf < T(0)) pk = fmin(pk, sdiv(klo - ki, dkf));
        if (dwf > T(0)) pw = fmin(pw, sdiv(whi - wi, dwf));
        else if (dwf < T(0)) pw = fmin(pw, sdiv(wlo - wi, dwf));
    }
    lg[0] = pk * g[4];
    lg[1] = pk * g[5];
    lg[2] = pw * g[6];
    lg[3] = pw * g[7];
    T cd = sdiv(T(2 * kSw2), wi) * (g[4] * g[6] + g[5] * g[7]);
    cd = cd > T(1e-20) ? cd : T(1e-20);
    const T a = sdiv(sqrt(ki), T(kBstar) * wi * di);
    const T bb = sdiv(T(500) * nu, wi * di * di);
    const T c = sdiv(T(4 * kSw2) * ki, cd * di * di);
    const T arg1 = fmin(fmax(a, bb), c);
    const T a2 = arg1 * arg1;
    f1 = tanh(a2 * a2);
}

// Face data of the k / omega update for one face: the neighbour's (u, v, k, omega), its
// limited k / omega gradients, f1 and nu_t; or the boundary values.
template <class T>
struct SstFace {
    bool has, bnd;
    T u, v, k, w;        // neighbour or boundary values
    T lg[4];             // neighbour limited gradients (interior only)
    T gn[4];             // neighbour gradients of k, omega (non-orthogonal correction only)
    T f1, nut;           // neighbour (interior only)
    T snx, sny, rox, roy, rnx, rny, dinv;
};

// Convection (limited second-order upwind, mean face velocity), central diffusion (mean face
// coefficient), explicit production and cross diffusion, point-implicit destruction; then f2,
// nu_t = a1 k / max(a1 omega, S f2) and tau = (nu + nu_t)/cs^2.
// The own-cell gradient enters the update only through three invariants: S_ij S_ij, div u and
// grad k . grad omega (Sec. 2: production, nu_t limiter, cross diffusion).
template <class T>
__device__ __forceinline__ void sst_invariants(const T *g, T &SS, T &dv, T &kw) {
    const T s11 = g[0], s22 = g[3], s12 = T(0.5) * (g[1] + g[2]);
    SS = s11 * s11 + s22 * s22 + T(2) * s12 * s12;
    dv = s11 + s22;
    kw = g[4] * g[6] + g[5] * g[7];
}

// g (the own gradients) is read by the reading variants only; SS, dv, kw are its invariants.
template <class T, bool NONORTH>
__device__ __forceinline__ void sst_cell_update(const InstParam &P, T dt, T ui, T vi, T ki, T wi,
                                                T nti, T di, const T *g, T SS, T dv, T kw,
                                                const T *lgi, T f1, const SstFace<T> *F, T &kn,
                                                T &wn, T &ntn, T &tnew) {
    const T nu = ipv<T>(P.nu, P.nu_f);
    const T sk_i = f1 * T(kSk1) + (T(1) - f1) * T(kSk2);
    const T sw_i = f1 * T(kSw1) + (T(1) - f1) * T(kSw2);
    T ck = 0, cw = 0, dk = 0, dw = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const SstFace<T> &f = F[m];
        if (!f.has) continue;
        const T kin = ki + lgi[0] * f.rox + lgi[1] * f.roy;
        const T win = wi + lgi[2] * f.rox + lgi[3] * f.roy;
        const T dla = sqrt(f.snx * f.snx + f.sny * f.sny);  // |n dl / A| -> dl / A
        if (!f.bnd) {
            const T uf = T(0.5) * (ui + f.u), vf = T(0.5) * (vi + f.v);
            const T un = uf * f.snx + vf * f.sny;  // (u_f . n) dl / A
            T kup, wup;
            if (un >= T(0)) {
                kup = kin; wup = win;
            } else {
                kup = f.k + f.lg[0] * f.rnx + f.lg[1] * f.rny;
                wup = f.w + f.lg[2] * f.rnx + f.lg[3] * f.rny;
            }
            const T skj = f.f1 * T(kSk1) + (T(1) - f.f1) * T(kSk2);
            const T swj = f.f1 * T(kSw1) + (T(1) - f.f1) * T(kSw2);
            const T gkf = T(0.5) * ((nu + sk_i * nti) + (nu + skj * f.nut));
            const T gwf = T(0.5) * ((nu + sw_i * nti) + (nu + swj * f.nut));
            ck += un * kup;
            cw += un * wup;
            T dkn = (f.k - ki) * f.dinv, dwn = (f.w - wi) * f.dinv;
            if (NONORTH && (P.variant & 2)) {
                // non-orthogonal correction (reading variant 2): + mean grad . (n - d/|d|),
                // d = x_j - x_i = r_own - r_nbr, n the unit face normal
                const T tx = f.snx / dla - (f.rox - f.rnx) * f.dinv;
                const T ty = f.sny / dla - (f.roy - f.rny) * f.dinv;
                dkn += T(0.5) * ((g[4] + f.gn[0]) * tx + (g[5] + f.gn[1]) * ty);
                dwn += T(0.5) * ((g[6] + f.gn[2]) * tx + (g[7] + f.gn[3]) * ty);
            }
            dk += gkf * dkn * dla;
            dw += gwf * dwn * dla;
        } else {
            const T un = f.u * f.snx + f.v * f.sny;
            const T kup = un >= T(0) ? kin : f.k;
            const T wup = un >= T(0) ? win : f.w;
            ck += un * kup;
            cw += un * wup;
            T dkn = (f.k - ki) * f.dinv, dwn = (f.w - wi) * f.dinv;
            if (NONORTH && (P.variant & 2)) {  // d = r_own (face midpoint - centroid)
                const T tx = f.snx / dla - f.rox * f.dinv, ty = f.sny / dla - f.roy * f.dinv;
                dkn += g[4] * tx + g[5] * ty;
                dwn += g[6] * tx + g[7] * ty;
            }
            dk += (nu + sk_i * nti) * dkn * dla;
            dw += (nu + sw_i * nti) * dwn * dla;
        }
    }
    const T Sabs = sqrt(T(2) * SS);
    const T cw1 = T(kB1 / kBstar - kSw1 * kKappa * kKappa / 0.3);
    const T cw2 = T(kB2 / kBstar - kSw2 * kKappa * kKappa / 0.3);
    const T gam = f1 * cw1 + (T(1) - f1) * cw2;
    T pk = nti * (T(2) * SS - T(2.0 / 3.0) * dv * dv) - T(2.0 / 3.0) * ki * dv;
    if (NONORTH && (P.variant & 8)) {  // Menter's production limiter (reading variant 8)
        const T cap = T(10.0 * kBstar) * wi * ki;
        pk = pk > cap ? cap : pk;
    }
    T pw = gam * (T(2) * SS - T(2.0 / 3.0) * dv * dv);
    if (nti > T(0)) pw -= T(2.0 / 3.0) * gam * ki * dv / nti;
    const T cross = T(2) * (T(1) - f1) * T(kSw2) / wi * kw;
    const T rk = -ck + dk + pk;
    const T rw = -cw + dw + pw + cross;
    const T beta = f1 * T(kB1) + (T(1) - f1) * T(kB2);
    kn = (ki + dt * rk) / (T(1) + dt * T(kBstar) * wi);
    wn = (wi + dt * rw) / (T(1) + dt * beta * wi);
    kn = kn > T(0) ? kn : T(0);
    wn = wn > ipv<T>(P.omega_min, P.omega_min_f) ? wn : ipv<T>(P.omega_min, P.omega_min_f);
    const T arg2 = fmax(T(2) * sqrt(kn) / (T(kBstar) * wn * di), T(500) * nu / (wn * di * di));
    const T f2 = tanh(arg2 * arg2);
    ntn = T(kA1) * kn / fmax(T(kA1) * wn, Sabs * f2);
    tnew = (nu + ntn) / T(kCs2);
}

// ---- two-pass SST kernels (one thread per cell, neighbours gathered from global memory)
// Gradients of u, v, k, omega, the limited k / omega gradients and f1.
// Face geometry of cell i from the compact arrays (node positions gq, offsets d): face offset
// r_m, outward n dl / A, neighbour offset r_m - d_m, 1 / |d_m| and the least-squares weights.
template <class T>
__device__ __forceinline__ void compact_face_geo(const CompactGeo<T> &CG, size_t np, int i,
                                                 const bool *has, T *R, T *SN, T *RN, T *DI,
                                                 T *W) {
    T q[8], d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        q[k] = CG.gq[k * np + i];
        d[k] = CG.dv[k * np + i];
    }
    const bool tri = !has[3];
    auto end_x = [&](int m) { return m == 3 ? q[0] : (m == 2 && tri ? q[0] : q[2 * m + 2]); };
    auto end_y = [&](int m) { return m == 3 ? q[1] : (m == 2 && tri ? q[1] : q[2 * m + 3]); };
    T a2x = T(0), mxx = 0, mxy = 0, myy = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (m < 3 || !tri) a2x += q[2 * m] * end_y(m) - end_x(m) * q[2 * m + 1];
        if (has[m]) {
            mxx += d[2 * m] * d[2 * m];
            mxy += d[2 * m] * d[2 * m + 1];
            myy += d[2 * m + 1] * d[2 * m + 1];
        }
    }
    const T inv_a = a2x > T(0) ? T(2) / a2x : T(0);
    const T idet = T(1) / (mxx * myy - mxy * mxy);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const T x1 = end_x(m), y1 = end_y(m);
        R[2 * m] = T(0.5) * (q[2 * m] + x1);
        R[2 * m + 1] = T(0.5) * (q[2 * m + 1] + y1);
        SN[2 * m] = (y1 - q[2 * m + 1]) * inv_a;
        SN[2 * m + 1] = -(x1 - q[2 * m]) * inv_a;
        RN[2 * m] = R[2 * m] - d[2 * m];
        RN[2 * m + 1] = R[2 * m + 1] - d[2 * m + 1];
        DI[m] = has[m] ? T(1) / sqrt(d[2 * m] * d[2 * m] + d[2 * m + 1] * d[2 * m + 1]) : T(0);
        W[2 * m] = (myy * d[2 * m] - mxy * d[2 * m + 1]) * idet;
        W[2 * m + 1] = (mxx * d[2 * m + 1] - mxy * d[2 * m]) * idet;
    }
}

// Packed per-cell SST records of the fused path, written by the gradient kernel and gathered
// by the update kernel for every neighbour: rec8 = (u, v, k, omega, limited grad k, limited
// grad omega) in one 32-byte (FP32) row and rec2 = (f1, nu_t), so that a neighbour costs
// three vector loads instead of ten scattered ones.
template <class T>
__device__ __forceinline__ void sst_store_rec(T *__restrict__ rec8, T *__restrict__ rec2, int i, const T *v8,
                                              T f1, T nut) {
    T *r = rec8 + 8 * static_cast<size_t>(i);
    if constexpr (std::is_same<T, float>::value) {
        *reinterpret_cast<float4 *>(r) = make_float4(v8[0], v8[1], v8[2], v8[3]);
        *reinterpret_cast<float4 *>(r + 4) = make_float4(v8[4], v8[5], v8[6], v8[7]);
        *reinterpret_cast<float2 *>(rec2 + 2 * static_cast<size_t>(i)) = make_float2(f1, nut);
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) r[c] = v8[c];
        rec2[2 * static_cast<size_t>(i)] = f1;
        rec2[2 * static_cast<size_t>(i) + 1] = nut;
    }
}
template <class T>
__device__ __forceinline__ void sst_load_rec(const T *__restrict__ rec8, const T *__restrict__ rec2, int i, T *v8,
                                             T &f1, T &nut) {
    const T *r = rec8 + 8 * static_cast<size_t>(i);
    if constexpr (std::is_same<T, float>::value) {
        const float4 a = *reinterpret_cast<const float4 *>(r), b = *reinterpret_cast<const float4 *>(r + 4);
        v8[0] = a.x; v8[1] = a.y; v8[2] = a.z; v8[3] = a.w;
        v8[4] = b.x; v8[5] = b.y; v8[6] = b.z; v8[7] = b.w;
        const float2 c = *reinterpret_cast<const float2 *>(rec2 + 2 * static_cast<size_t>(i));
        f1 = c.x;
        nut = c.y;
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) v8[c] = r[c];
        f1 = rec2[2 * static_cast<size_t>(i)];
        nut = rec2[2 * static_cast<size_t>(i) + 1];
    }
}

// Both SST kernels run over one contiguous run of SST tiles per launch (tile0 + block; a
// laminar instance keeps tau = nu / cs^2 and is not visited), so a thread issues the loads of
// its own cell at once, without waiting for the instance parameters first.
template <class T, bool COMPACT>
__global__ void __launch_bounds__(kTile)
    k_sst_grad(const T *__restrict__ mac, const T *__restrict__ kk, const T *__restrict__ ww,
               T *__restrict__ grads, T *__restrict__ f1out, Geo<T> G, CompactGeo<T> CG,
               const T *__restrict__ nut, T *__restrict__ rec8, T *__restrict__ rec2, bool inv_only,
               int tile0) {
    const int tile = tile0 + static_cast<int>(blockIdx.x);
    const int i = tile * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[tile]];
    const T nu = ipv<T>(P.nu, P.nu_f);
    const T own[4] = {mac[np + i], mac[2 * np + i], kk[i], ww[i]};
    const T di = G.wdist[i];
    bool has[4];
    int nbs[4];
    T q[4][4], W[8], R[8];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        nbs[m] = G.nbr[m * np + i];
        has[m] = nbs[m] != kNone;
    }
    // The least-squares weights are read as precomputed (formed in FP64 on the host): on
    // the 1000:1 wall cells of y+ ~ 1 meshes M = sum d d^T has a condition number near 1e7, and
    // inverting it in FP32 on chip would leave the weights with almost no correct digits.
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        W[2 * m] = G.lsq[(2 * m) * np + i];
        W[2 * m + 1] = G.lsq[(2 * m + 1) * np + i];
    }
    if (COMPACT) {  // face offsets from the node positions
        T q8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) q8[k] = CG.gq[k * np + i];
        const bool tri = !has[3];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const T x1 = m == 3 ? q8[0] : (m == 2 && tri ? q8[0] : q8[2 * m + 2]);
            const T y1 = m == 3 ? q8[1] : (m == 2 && tri ? q8[1] : q8[2 * m + 3]);
            R[2 * m] = T(0.5) * (q8[2 * m] + x1);
            R[2 * m + 1] = T(0.5) * (q8[2 * m + 1] + y1);
        }
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            R[2 * m] = G.rown[(2 * m) * np + i];
            R[2 * m + 1] = G.rown[(2 * m + 1) * np + i];
        }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int nb = nbs[m];
        if (nb == kNone) continue;
        if (nb >= 0) {
            q[m][0] = mac[np + nb]; q[m][1] = mac[2 * np + nb]; q[m][2] = kk[nb]; q[m][3] = ww[nb];
        } else {
            sst_bvals(G, -nb - 1, nu, own[0], own[1], own[2], own[3], di, q[m][0], q[m][1], q[m][2],
                      q[m][3]);
        }
    }
    T g[8], lg[4], f1;
    sst_cell_grad(own[2], own[3], di, nu, has, q, W, R, own, g, lg, f1);
    if (inv_only) {  // the update needs the invariants of the own gradient only
        T SS, dv, kw;
        sst_invariants(g, SS, dv, kw);
        grads[i] = SS;
        grads[np + i] = dv;
        grads[2 * np + i] = kw;
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) grads[c * np + i] = g[c];
    }
    if (rec8 != nullptr) {  // fused path: the packed record the update gathers
        const T v8[8] = {own[0], own[1], own[2], own[3], lg[0], lg[1], lg[2], lg[3]};
        sst_store_rec(rec8, rec2, i, v8, f1, nut[i]);
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) grads[(8 + c) * np + i] = lg[c];
        f1out[i] = f1;
    }
}

// The k / omega update and the new relaxation time (and, on the fused path, f^(1)).  In
// float, 5 blocks of 128 per SM (96 registers, a few spilled) run faster than 4 (120).
// NONORTH compiles the SST reading variants in (2: non-orthogonal diffusion correction, 8:
// production limiter); without them the kernel keeps the register count (and occupancy) of
// the default reading.
template <class T, bool COMPACT, bool NONORTH>
__global__ void __launch_bounds__(kTile, sizeof(T) == 4 ? 5 : 1)
    k_sst_update(const T *__restrict__ mac, const T *__restrict__ kk, const T *__restrict__ ww,
                 const T *__restrict__ nut, const T *__restrict__ grads,
                 const T *__restrict__ f1a, T *__restrict__ k_out, T *__restrict__ w_out,
                 T *__restrict__ nut_out, T *__restrict__ tau, Geo<T> G,
                 const T *__restrict__ fn, T *__restrict__ frel, CompactGeo<T> CG,
                 const T *__restrict__ rec8, const T *__restrict__ rec2, int tile0) {
    const int tile = tile0 + static_cast<int>(blockIdx.x);
    const int i = tile * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[tile]];
    const T nu = ipv<T>(P.nu, P.nu_f);
    const bool packed = COMPACT && rec8 != nullptr;
    T ui, vi, ki, wi, nti, f1i;
    T g[8], lgi[4];
    if (packed) {
        T v8[8];
        sst_load_rec(rec8, rec2, i, v8, f1i, nti);
        ui = v8[0]; vi = v8[1]; ki = v8[2]; wi = v8[3];
#pragma unroll
        for (int c = 0; c < 4; ++c) lgi[c] = v8[4 + c];
    } else {
        ui = mac[np + i]; vi = mac[2 * np + i]; ki = kk[i]; wi = ww[i]; nti = nut[i];
        f1i = f1a[i];
#pragma unroll
        for (int c = 0; c < 4; ++c) lgi[c] = grads[(8 + c) * np + i];
    }
    const T di = G.wdist[i];
    T SS, dv, kw;
    if (packed && !NONORTH) {  // the grad kernel stored the invariants alone
        SS = grads[i];
        dv = grads[np + i];
        kw = grads[2 * np + i];
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) g[c] = grads[c * np + i];
        sst_invariants(g, SS, dv, kw);
    }
    SstFace<T> F[4];
    int nbs[4];
    bool has[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        nbs[m] = G.nbr[m * np + i];
        has[m] = nbs[m] != kNone;
    }
    T R[8], SN[8], RN[8], DI[4];
    if (COMPACT) {
        T W[8];
        compact_face_geo(CG, np, i, has, R, SN, RN, DI, W);
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (!has[m]) continue;
            SN[2 * m] = G.sn[(2 * m) * np + i]; SN[2 * m + 1] = G.sn[(2 * m + 1) * np + i];
            R[2 * m] = G.rown[(2 * m) * np + i]; R[2 * m + 1] = G.rown[(2 * m + 1) * np + i];
            RN[2 * m] = G.rnbr[(2 * m) * np + i]; RN[2 * m + 1] = G.rnbr[(2 * m + 1) * np + i];
            DI[m] = G.dinv[m * np + i];
        }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int nb = nbs[m];
        SstFace<T> &f = F[m];
        f.has = has[m];
        if (!f.has) continue;
        f.bnd = nb < 0;
        f.snx = SN[2 * m]; f.sny = SN[2 * m + 1];
        f.rox = R[2 * m]; f.roy = R[2 * m + 1];
        f.dinv = DI[m];
        if (nb >= 0) {
            f.rnx = RN[2 * m]; f.rny = RN[2 * m + 1];
            if (packed) {
                T v8[8];
                sst_load_rec(rec8, rec2, nb, v8, f.f1, f.nut);
                f.u = v8[0]; f.v = v8[1]; f.k = v8[2]; f.w = v8[3];
#pragma unroll
                for (int c = 0; c < 4; ++c) f.lg[c] = v8[4 + c];
            } else {
                f.u = mac[np + nb]; f.v = mac[2 * np + nb]; f.k = kk[nb]; f.w = ww[nb];
#pragma unroll
                for (int c = 0; c < 4; ++c) f.lg[c] = grads[(8 + c) * np + nb];
                f.f1 = f1a[nb];
                f.nut = nut[nb];
            }
            if (NONORTH && (P.variant & 2)) {
#pragma unroll
                for (int c = 0; c < 4; ++c) f.gn[c] = grads[(4 + c) * np + nb];
            }
        } else {
            sst_bvals(G, -nb - 1, nu, ui, vi, ki, wi, di, f.u, f.v, f.k, f.w);
        }
    }
    T kn, wn, ntn, tnew;
    const T dt_i = cell_dt(G, P, i);
    sst_cell_update<T, NONORTH>(P, dt_i, ui, vi, ki, wi, nti, di, g, SS, dv, kw, lgi, f1i, F, kn, wn, ntn,
                                tnew);
    k_out[i] = kn;
    w_out[i] = wn;
    nut_out[i] = ntn;
    tau[i] = tnew;
    if (frel != nullptr) {  // fused path: stage 1's f^(1) with the new relaxation time
        T f[kQ];
        load9(fn, np, i, f);
        relax9(f, ipv<T>(P.rho0, P.rho0_f), dt_i, tnew);
        store9(frel, np, i, f);
    }
}

// ------------------------------------------------------------------ state I/O kernels
template <class T>
__global__ void k_init_state(T *__restrict__ fn, T *__restrict__ mac, const double *__restrict__ r0,
                             const double *__restrict__ u0, const double *__restrict__ v0,
                             Geo<T> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam &P = G.ip[G.tile_inst[blockIdx.x]];
    const T rho0 = ipv<T>(P.rho0, P.rho0_f);
    const T r = T(r0[i]), u = T(u0[i]), v = T(v0[i]);
    T eq[kQ];
    feq_dev(T(r0[i] - double(rho0)), r, u, v, eq);
    store9(fn, np, i, eq);
    T dr, rr, uu, vv;
    moments(eq, rho0, dr, rr, uu, vv);
    mac[i] = rr;
    mac[np + i] = uu;
    mac[2 * np + i] = vv;
}

// out[perm[k] * 9 + a] = f[a][off + k] + w_a rho0   (k < nc)
template <class T>
__global__ void k_gather_f(const T *__restrict__ f, const int *__restrict__ perm, int off, int nc,
                           double rho0, size_t np, double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const int dst = perm[k];
    for (int a = 0; a < kQ; ++a) {
        const double wa = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        out[static_cast<size_t>(dst) * kQ + a] = double(f[a * np + off + k]) + wa * rho0;
    }
}

// Per wall face momentum flux and Cp (FP64): out[5][nb_inst] = fx, fy, cp, dfx/dp, dfy/dp (the
// last two are 0 except for the tangent type).
template <class T>
__global__ void k_wall_forces(const T *__restrict__ fn, const int *__restrict__ bowner,
                             const T *__restrict__ bnrm, const T *__restrict__ blen, int b0,
                             int nbi, double rho0, double uref, Geo<T> G,
                             double *__restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nbi) return;
    const int b = b0 + q;
    const size_t np = G.np;
    out[q] = out[nbi + q] = out[2 * nbi + q] = out[3 * nbi + q] = out[4 * nbi + q] = 0.0;
    if (G.btype[b] != FVLBM_BC_WALL) return;
    const int i = bowner[b];
    T fi[kQ], fb[kQ], dr, r, u, v;
    load9(fn, np, i, fi);
    moments(fi, T(rho0), dr, r, u, v);
    const T nx = bnrm[b], ny = bnrm[G.nbt + b];
    boundary_values(G.btype[b], G.bval + b, 0, G.nbt, nx, ny, fi, dr, r, u, v, T(rho0), fb);
    double fx = 0, fy = 0, dfx = 0, dfy = 0;
    for (int a = 0; a < kQ; ++a) {
        const double en = double(ex_of(a)) * double(nx) + double(ey_of(a)) * double(ny);
        const double wa = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        const double m = en * (double(fb[a]) + wa * rho0) * double(blen[b]);
        // derivative: f_bc, the normal and the length may all depend on p
        const double dm = tangent_of((T(ex_of(a)) * nx + T(ey_of(a)) * ny) * (fb[a] + T(wa * rho0)) * blen[b]);
        fx += ex_of(a) * m;
        fy += ey_of(a) * m;
        dfx += ex_of(a) * dm;
        dfy += ey_of(a) * dm;
    }
    out[q] = fx;
    out[nbi + q] = fy;
    out[3 * nbi + q] = dfx;
    out[4 * nbi + q] = dfy;
    out[2 * nbi + q] = (kCs2 * double(r) - kCs2 * rho0) / (0.5 * rho0 * uref * uref);
}

// All instances at once: output position j (instances concatenated in input order, cells in
// input order within each) maps to internal cell map[j].
template <class T>
__global__ void k_gather_f_all(const T *__restrict__ f, const int *__restrict__ map, int total,
                               size_t np, const int *__restrict__ tile_inst,
                               const InstParam *__restrict__ ip, double *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= total) return;
    const int i = map[j];
    const double rho0 = ip[tile_inst[i / kTile]].rho0;
    for (int a = 0; a < kQ; ++a) {
        const double wa = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        out[static_cast<size_t>(j) * kQ + a] = double(f[a * np + i]) + wa * rho0;
    }
}

// State input: internal cells [i0, i0 + n), each reading its record at input position
// inv[i] - po of the concatenated input order (padding cells: inv = -1, left as they are).
// IN = double: absolute f; IN = float: the FP32 deviation f - w_alpha rho0.  Writes f^n, the
// macros and f^(1) of the coming step (relaxed like k_stage1, for the fused stages).
template <class T, class IN>
__global__ void k_scatter_state(T *__restrict__ f, T *__restrict__ mac, T *__restrict__ frel,
                                const T *__restrict__ tau, const int *__restrict__ inv, int i0, int n,
                                int po, Geo<T> G, const IN *__restrict__ in) {
    // one thread per internal cell i (the state arrays are written coalesced; the input record
    // of the cell, 9 consecutive values, is read where the input order puts it)
    const int i = i0 + static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= i0 + n) return;
    const int jo = inv[i];
    if (jo < 0) return;  // padding cell of a tile
    const size_t j = static_cast<size_t>(jo - po);
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[i / kTile]];
    T d[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        if constexpr (sizeof(IN) == sizeof(double)) {
            const double wa = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
            d[a] = T(double(in[j * kQ + a]) - wa * P.rho0);
        } else if constexpr (std::is_same<T, float>::value) {
            d[a] = in[j * kQ + a];  // the deviation itself, with no round trip through double
        } else {
            d[a] = T(double(in[j * kQ + a]));
        }
        f[a * np + i] = d[a];
    }
    T dr, r, u, v;
    moments(d, ipv<T>(P.rho0, P.rho0_f), dr, r, u, v);
    mac[i] = r;
    mac[np + i] = u;
    mac[2 * np + i] = v;
    if (frel != nullptr) {  // f^(1) of the coming step, for the forms that stage it
        relax9(d, ipv<T>(P.rho0, P.rho0_f), cell_dt(G, P, i), tau[i]);
        store9(frel, np, i, d);
    }
}

// The same for a list of cells: position j < n of the input takes internal cell map[j] (the
// cell lists of fvlbm_set_cells).
template <class T, class IN>
__global__ void k_scatter_list(T *__restrict__ f, T *__restrict__ mac, T *__restrict__ frel,
                               const T *__restrict__ tau, const int *__restrict__ map, int n,
                               Geo<T> G, const IN *__restrict__ in) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int i = map[j];
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[i / kTile]];
    T d[kQ];
    for (int a = 0; a < kQ; ++a) {
        const double x = double(in[static_cast<size_t>(j) * kQ + a]);
        if (sizeof(IN) == sizeof(double)) {
            const double wa = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
            d[a] = T(x - wa * P.rho0);
        } else {
            d[a] = T(x);
        }
        f[a * np + i] = d[a];
    }
    T dr, r, u, v;
    moments(d, ipv<T>(P.rho0, P.rho0_f), dr, r, u, v);
    mac[i] = r;
    mac[np + i] = u;
    mac[2 * np + i] = v;
    if (frel != nullptr) {
        relax9(d, ipv<T>(P.rho0, P.rho0_f), cell_dt(G, P, i), tau[i]);
        store9(frel, np, i, d);
    }
}

// Cell lists of one instance (halo exchange of a partitioned mesh): map[j] = the internal id
// of input cell cells[j] of the instance (amap: input id -> internal id, from the instance's
// first cell).
__global__ void k_cell_map(const int *__restrict__ amap, const int *__restrict__ cells, int n,
                           int *__restrict__ map) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) map[j] = amap[cells[j]];
}

// out_f[j][9] = f of cell map[j] (absolute: deviation + w_alpha rho0); k, omega, nu_t of the
// current ping-pong buffers into out_t[3][n] when kk is given.
template <class T>
__global__ void k_get_cells(const T *__restrict__ f, const T *__restrict__ kk, const T *__restrict__ ww,
                            const T *__restrict__ nut, const int *__restrict__ map, int n, double rho0,
                            size_t np, double *__restrict__ out_f, double *__restrict__ out_t) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int i = map[j];
    for (int a = 0; a < kQ; ++a) {
        const double wa = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        out_f[static_cast<size_t>(j) * kQ + a] = value_of(f[a * np + i]) + wa * rho0;
    }
    if (kk != nullptr) {
        out_t[j] = value_of(kk[i]);
        out_t[n + j] = value_of(ww[i]);
        out_t[2 * n + j] = value_of(nut[i]);
    }
}

// k, omega, nu_t of cell map[j] from in[3][n] (into the current ping-pong buffers).
template <class T>
__global__ void k_set_turb(T *__restrict__ kk, T *__restrict__ ww, T *__restrict__ nut,
                           const int *__restrict__ map, int n, const double *__restrict__ in) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int i = map[j];
    kk[i] = T(in[j]);
    ww[i] = T(in[n + j]);
    nut[i] = T(in[2 * n + j]);
}

// Wall distance of cell map[j] from in[j].
template <class T>
__global__ void k_set_wdist(T *__restrict__ wdist, const int *__restrict__ map, int n,
                            const double *__restrict__ in) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) wdist[map[j]] = T(in[j]);
}

// Ghost exchange of a split mesh on device buffers: row j of vals (kXRow doubles) holds cell
// map[j]'s f (absolute: deviation + w_alpha rho0), k, omega, nu_t (current buffers).
template <class T>
__global__ void k_pack_cells(const T *__restrict__ f, const T *__restrict__ kk, const T *__restrict__ ww,
                             const T *__restrict__ nut, const int *__restrict__ map, int n, Geo<T> G,
                             double *__restrict__ vals) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int i = map[j];
    const size_t np = G.np;
    const double rho0 = G.ip[G.tile_inst[i / kTile]].rho0;
    double *v = vals + static_cast<size_t>(j) * kXRow;
    for (int a = 0; a < kQ; ++a) {
        const double wa = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        v[a] = value_of(f[a * np + i]) + wa * rho0;
    }
    v[9] = value_of(kk[i]);
    v[10] = value_of(ww[i]);
    v[11] = value_of(nut[i]);
}

// The reverse: f^n (deviation), the macros and, where kept, f^(1) of the coming step (as
// fvlbm_set_f writes them), k, omega and nu_t of cell map[j] from row j of vals.
template <class T>
__global__ void k_unpack_cells(T *__restrict__ f, T *__restrict__ mac, T *__restrict__ frel,
                               const T *__restrict__ tau, T *__restrict__ kk, T *__restrict__ ww,
                               T *__restrict__ nut, const int *__restrict__ map, int n, Geo<T> G,
                               const double *__restrict__ vals) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int i = map[j];
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[i / kTile]];
    const double *v = vals + static_cast<size_t>(j) * kXRow;
    T d[kQ];
    for (int a = 0; a < kQ; ++a) {
        const double wa = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        d[a] = T(v[a] - wa * P.rho0);
        f[a * np + i] = d[a];
    }
    T dr, r, u, w;
    moments(d, ipv<T>(P.rho0, P.rho0_f), dr, r, u, w);
    mac[i] = r;
    mac[np + i] = u;
    mac[2 * np + i] = w;
    kk[i] = T(v[9]);
    ww[i] = T(v[10]);
    nut[i] = T(v[11]);
    if (frel != nullptr) {
        relax9(d, ipv<T>(P.rho0, P.rho0_f), cell_dt(G, P, i), tau[i]);
        store9(frel, np, i, d);
    }
}

// Output fields[q][j] for the fields q (rho, u, v, k, omega, nu_t) selected by mask bit q.
template <class T>
__global__ void k_gather_fields_map(const T *__restrict__ mac, const T *__restrict__ kk,
                                    const T *__restrict__ ww, const T *__restrict__ nut,
                                    const int *__restrict__ map, int n, size_t np, unsigned mask,
                                    double *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int i = map[j];
    const size_t m = n;
    if (mask & 1u) out[0 * m + j] = double(mac[i]);
    if (mask & 2u) out[1 * m + j] = double(mac[np + i]);
    if (mask & 4u) out[2 * m + j] = double(mac[2 * np + i]);
    if (mask & 8u) out[3 * m + j] = double(kk[i]);
    if (mask & 16u) out[4 * m + j] = double(ww[i]);
    if (mask & 32u) out[5 * m + j] = double(nut[i]);
}

template <class T>
__global__ void k_gather_fdev32(const T *__restrict__ f, const int *__restrict__ map, int n, size_t np,
                                float *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int i = map[j];
    for (int a = 0; a < kQ; ++a) out[static_cast<size_t>(j) * kQ + a] = float(double(f[a * np + i]));
}

// Tangent seed: df/dp of instance cells (off + k) from in[perm[k] * 9 + a]; the macros are
// recomputed from the seeded f so that their derivatives agree.
__global__ void k_seed_df(Dual *__restrict__ f, Dual *__restrict__ mac, const int *__restrict__ perm,
                          int off, int nc, double rho0, size_t np, const double *__restrict__ in) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const int src = perm[k];
    Dual d[kQ];
    for (int a = 0; a < kQ; ++a) {
        d[a] = f[a * np + off + k];
        d[a].d = in[static_cast<size_t>(src) * kQ + a];
        f[a * np + off + k] = d[a];
    }
    Dual dr, r, u, v;
    moments(d, Dual(rho0), dr, r, u, v);
    mac[off + k] = r;
    mac[np + off + k] = u;
    mac[2 * np + off + k] = v;
}

__global__ void k_gather_df(const Dual *__restrict__ f, const int *__restrict__ perm, int off, int nc,
                            size_t np, double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const int dst = perm[k];
    for (int a = 0; a < kQ; ++a) out[static_cast<size_t>(dst) * kQ + a] = f[a * np + off + k].d;
}

}  // namespace fvlbm

// ==================================================================== handle and C ABI
using namespace fvlbm;

namespace {

// Copy of one instance's input mesh, kept by tangent handles so that the geometry can be
// differentiated with respect to node positions after create.
struct MeshCopy {
    std::vector<double> xy, bval, pshift;
    std::vector<int> cell_ptr, cell_nodes, bnodes, btype, ppairs, perm;
    fvlbm_params params{};
};

struct InstInfo {
    int nc, np, nb, n_bedges_in, sst, n_nodes;
    int cell_off, tile_off, bface_off;
    double dt, rho0, uref, lref, alpha_deg, nu;
    std::vector<int> bedge_of;   // boundary face -> input edge (local)
    std::shared_ptr<MeshCopy> mesh;  // FP64 and tangent handles (shape derivatives)
};

struct KernelTimer {
    std::string name;
    double ms = 0;
    int launches = 0;
};

}  // namespace

struct fvlbm_handle {
    int device = 0;
    int precision = FVLBM_FP64;
    bool sst = false;
    bool own_stream = false;
    cudaStream_t stream = nullptr;
    int np = 0, nbt = 0, ntiles = 0, ninst = 0;
    std::vector<InstInfo> inst;
    long long steps = 0;
    size_t device_bytes = 0;
    std::vector<void *> allocs;
    struct XList {           // ghost-exchange cell lists (fvlbm_set_exchange_list)
        int instance, n;
        int *d_map;          // internal ids
    };
    std::vector<XList> xlists;
    // device arrays (element type T = double or float; stored as void*)
    int *d_nbr = nullptr, *d_tile_inst = nullptr, *d_btype = nullptr, *d_bowner = nullptr;
    int *d_perm = nullptr, *d_inst_tile0 = nullptr;
    std::vector<int2> sst_runs;  // (first tile, tiles) of each contiguous run of SST instances
    int *d_all_map = nullptr;   // output position (all instances) -> internal cell
    int *d_all_inv = nullptr;   // internal cell -> output position (all instances), -1: padding
    int *d_back = nullptr;      // FP64 handles: slot of each face at its neighbour [4 np] (adjoint)
    size_t adj_budget = 0;      // device bytes the adjoint may keep stage values in (0: half the free)
    int total_nc = 0, total_nb = 0;
    // fused path: per-block halo lists and local adjacency, for each fused block size
    struct HaloSet {
        bool ok = false;
        int blk = 0, nblk = 0, emax = 0, gmax = 0;
        size_t smem = 0;
        int *d_halo_ptr = nullptr, *d_halo = nullptr, *d_r1 = nullptr, *d_adj_ptr = nullptr;
        int *d_inst_blk0 = nullptr;
        unsigned *d_adj = nullptr;
    } hs[2];                // [0]: 256-cell blocks, [1]: 128-cell blocks
    struct FvSet {          // work items of the face-value fused kernel (config 3)
        bool ok = false;
        int nitem = 0, n_split = 0, n_ovf = 0;  // items; blocks split; items using the overflow
        int4 *d_hdr = nullptr;
        int *d_halo = nullptr, *d_ovf = nullptr, *d_inst_item0 = nullptr;
        uint4 *d_adj = nullptr;
    } fv;
    bool fused = false;     // fused kernels available (IMEX scheme, kernel_path 0 or 2)
    int config = 2;         // 0: fused 256, 1: fused 128, 2: two-pass, 3: face-value fused
                            // (see fvlbm_autotune)
    int scheme = 0;         // 0: IMEX Runge-Kutta; 1: explicit Euler (comparison scheme)
    int kernel_path = 0;    // as requested at create (fvlbm_params.kernel_path)
    bool limit_f = false;   // an instance uses the limiter variant (two-pass kernels only)
    bool nonorth = false;   // an instance uses an SST reading variant (2 or 8)
    bool per_stage = false; // SST solved before every stage (reading variant 4; two-pass only)
    unsigned long long order_hash = 0;  // checksum of the internal cell order (state blobs)
    struct AsyncIO {
        bool init = false;
        cudaStream_t s_in = nullptr, s_out = nullptr;
        double *d_in[2] = {nullptr, nullptr}, *d_out[2] = {nullptr, nullptr};
        size_t in_cap[2] = {0, 0}, out_cap[2] = {0, 0};
        cudaEvent_t in_ready[2], in_free[2], out_ready[2], out_free[2];
        int in_next = 0, out_next = 0;
    } aio;
    int rollback_every = 0;             // watchdog: device copy of the state every N steps
    void *rollback = nullptr;           // that copy (state_regions layout)
    long long rollback_step = -1, rollback_last = -1;
    int rollback_turb = 0;
    void *tau1 = nullptr, *mac2 = nullptr;  // per-stage SST: tau of stage 1, stage macros
    int *d_err = nullptr;   // device error flag (a staging wait gave up)
    long long wait_first = kWaitLimit;  // polls of the fused kernels' first staging wait
    void *gq = nullptr;     // fused path: node positions minus centroid [8 np]
    void *geo16 = nullptr;  // face-value path: per cell q[8] then least-squares W[8] [np][16]
    void *dvec = nullptr;   // fused path: neighbour-centroid offsets d_m [8 np]
    InstParam *d_ip = nullptr;
    void *sn = nullptr, *lsq = nullptr, *rown = nullptr, *rnbr = nullptr, *dinv = nullptr;
    void *area = nullptr, *wdist = nullptr, *bval = nullptr, *bnrm = nullptr, *blen = nullptr;
    void *fn = nullptr, *s0 = nullptr, *s1 = nullptr, *bacc = nullptr, *cacc = nullptr;
    void *grad = nullptr, *tau = nullptr, *mac = nullptr;
    void *frel = nullptr;   // fused path: f^(1) of the coming step (relaxed f^n)
    void *dtc = nullptr;    // local time stepping: dt of each cell (NULL: every instance global)
    void *kk[2] = {nullptr, nullptr}, *ww[2] = {nullptr, nullptr}, *nut[2] = {nullptr, nullptr};
    void *sgrad = nullptr, *f1 = nullptr;
    void *sst_rec8 = nullptr, *sst_rec2 = nullptr;  // fused path: packed SST records [np][8], [np][2]
    int turb = 0;  // which of the k/omega/nu_t ping-pong buffers is current
    double *d_partial = nullptr, *d_inst_sums = nullptr, *d_io = nullptr;
    size_t io_bytes = 0;
    // [0]: 1 step (laminar); [1 + parity]: kGraphSteps steps starting from k/omega/nu_t
    // ping-pong parity 0 or 1 (laminar runs use [1] only)
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
    bool profiling = false;
    std::vector<KernelTimer> timers;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
};

namespace {

constexpr int kGraphSteps = 16;

// Runs f with a value of the element type of the handle's precision (double, float or the
// tangent Dual) so that one generic body serves every precision.
template <class F>
void dispatch(int precision, F &&f) {
    if (precision == FVLBM_FP64)
        f(double(0));
    else if (precision == FVLBM_FP32_DEV)
        f(float(0));
    else
        f(Dual());
}

// The fused stage kernels exist for double and float; the tangent type runs the two-pass kernels.
template <class T>
constexpr bool kHasFused = !std::is_same<T, Dual>::value;

int cuda_fail(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return FVLBM_ERR_OOM;
    return FVLBM_ERR_CUDA;
}

#define CK(x)                                       \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

template <class T>
Geo<T> geo_of(const fvlbm_handle *h) {
    Geo<T> G;
    G.nbr = h->d_nbr;
    G.sn = static_cast<const T *>(h->sn);
    G.lsq = static_cast<const T *>(h->lsq);
    G.rown = static_cast<const T *>(h->rown);
    G.rnbr = static_cast<const T *>(h->rnbr);
    G.dinv = static_cast<const T *>(h->dinv);
    G.area = static_cast<const T *>(h->area);
    G.wdist = static_cast<const T *>(h->wdist);
    G.tile_inst = h->d_tile_inst;
    G.ip = h->d_ip;
    G.btype = h->d_btype;
    G.bval = static_cast<const T *>(h->bval);
    G.dtc = static_cast<const T *>(h->dtc);
    G.np = h->np;
    G.nbt = h->nbt;
    return G;
}

int dalloc(fvlbm_handle *h, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return cuda_fail(e);
    h->allocs.push_back(*p);
    h->device_bytes += bytes;
    return FVLBM_OK;
}

// The device arrays that make up the state a step reads (everything else is scratch):
// f^n, f^(1) of the coming step, the macros, tau and both k / omega / nu_t ping-pong buffers.
std::vector<std::pair<void *, size_t>> state_regions(const fvlbm_handle *h) {
    size_t ts = 0;
    dispatch(h->precision, [&](auto z_) { ts = sizeof(z_); });
    const size_t np = h->np;
    std::vector<std::pair<void *, size_t>> st = {
        {h->fn, kQ * np * ts}, {h->frel, kQ * np * ts}, {h->mac, 3 * np * ts}, {h->tau, np * ts}};
    for (int b = 0; b < 2; ++b) {
        st.push_back({h->kk[b], np * ts});
        st.push_back({h->ww[b], np * ts});
        st.push_back({h->nut[b], np * ts});
    }
    return st;
}

size_t state_bytes(const fvlbm_handle *h) {
    size_t t = 0;
    for (auto &e : state_regions(h)) t += e.second;
    return t;
}

struct StateHeader {
    char magic[8];
    int version, precision, np, ninst, turb, pad;
    long long steps;
    unsigned long long order_hash;
    unsigned long long payload;
};

template <class T>
int upload_as(fvlbm_handle *h, void **dst, const std::vector<double> &src) {
    std::vector<T> tmp(src.begin(), src.end());
    int rc = dalloc(h, dst, tmp.size() * sizeof(T));
    if (rc) return rc;
    CK(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FVLBM_OK;
}

template <class V>
int upload_raw(fvlbm_handle *h, V **dst, const std::vector<V> &src) {
    int rc = dalloc(h, reinterpret_cast<void **>(dst), src.size() * sizeof(V));
    if (rc) return rc;
    CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice));
    return FVLBM_OK;
}

template <class F>
void launch_timed(fvlbm_handle *h, int id, const char *name, F &&fn) {
    if (h->profiling) {
        if (static_cast<int>(h->timers.size()) <= id) h->timers.resize(id + 1);
        h->timers[id].name = name;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, h->stream);
        fn();
        cudaEventRecord(b, h->stream);
        h->pending.push_back({id, {a, b}});
    } else {
        fn();
    }
}

// Launch helper: an NVTX range named after the kernel around every launch (visible to nsys /
// ncu range filters), and CUDA events around it when profiling.
template <class F>
void launch(fvlbm_handle *h, int id, const char *name, F &&fn) {
    nvtxRangePushA(name);
    launch_timed(h, id, name, fn);
    nvtxRangePop();
}

// NVTX range for the lifetime of a scope (entry points with several returns).
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
};

enum KernelId {
    K_SST_GRAD, K_SST_UPDATE, K_STAGE1, K_GRAD, K_FLUX1, K_FLUX2, K_FLUX3, K_REDUCE,
    K_FUSED1, K_FUSED2, K_FUSED3, K_EULER, K_MACROS
};

// The three fused stages with BLK-cell blocks (halo set S).
template <class T, int BLK>
void enqueue_fused(fvlbm_handle *h, bool stats, const fvlbm_handle::HaloSet &S) {
    Geo<T> G = geo_of<T>(h);
    cudaStream_t s = h->stream;
    T *fn = static_cast<T *>(h->fn), *s0 = static_cast<T *>(h->s0), *s1 = static_cast<T *>(h->s1);
    T *B = static_cast<T *>(h->bacc), *C = static_cast<T *>(h->cacc);
    T *tau = static_cast<T *>(h->tau), *mac = static_cast<T *>(h->mac);
    T *fr = static_cast<T *>(h->frel);
    const Halo H{S.d_halo_ptr, S.d_halo, S.d_r1, S.d_adj_ptr, S.d_adj, h->d_err, S.emax, S.gmax,
                 h->wait_first};
    const CompactGeo<T> CG{static_cast<const T *>(h->gq), static_cast<const T *>(h->dvec)};
    const dim3 fg(S.nblk), fb(BLK);
    const size_t sm = S.smem;
    launch(h, K_FUSED1, "fused_stage1", [&] {
        k_fused_stage<T, 1, false, BLK><<<fg, fb, sm, s>>>(fr, s1, fn, B, C, tau, mac, nullptr, G, H, fr, CG);
    });
    launch(h, K_FUSED2, "fused_stage2", [&] {
        k_fused_stage<T, 2, false, BLK><<<fg, fb, sm, s>>>(s1, s0, fn, B, C, tau, mac, nullptr, G, H, fr, CG);
    });
    if (stats) {
        launch(h, K_FUSED3, "fused_stage3", [&] {
            k_fused_stage<T, 3, true, BLK><<<fg, fb, sm, s>>>(s0, s1, fn, B, C, tau, mac, h->d_partial, G, H, fr,
                                                              CG);
        });
        launch(h, K_REDUCE, "reduce", [&] {
            k_reduce_instances<<<h->ninst, kTile, 0, s>>>(h->d_partial, S.d_inst_blk0, h->d_inst_sums);
        });
    } else {
        launch(h, K_FUSED3, "fused_stage3", [&] {
            k_fused_stage<T, 3, false, BLK><<<fg, fb, sm, s>>>(s0, s1, fn, B, C, tau, mac, nullptr, G, H, fr, CG);
        });
    }
}

// The three stages in the face-value form (config 3): stage 1 reads f^n and writes f^(2) in
// cell-major rows into s1, stage 2 reads them and writes f^(3) likewise into s0.
// The three face-value stages over items [item0, item0 + nitem) on stream s; with stats,
// stage 3 also writes the items' FP64 partial sums (the caller reduces them).
template <class T>
void fv_stages(fvlbm_handle *h, bool stats, int item0, int nitem, cudaStream_t s) {
    Geo<T> G = geo_of<T>(h);
    T *fn = static_cast<T *>(h->fn), *s0 = static_cast<T *>(h->s0), *s1 = static_cast<T *>(h->s1);
    T *B = static_cast<T *>(h->bacc), *C = static_cast<T *>(h->cacc);
    T *tau = static_cast<T *>(h->tau), *mac = static_cast<T *>(h->mac);
    const FvItems W{h->fv.d_hdr, h->fv.d_halo, h->fv.d_ovf, h->fv.d_adj, h->d_err, h->wait_first, item0};
    const T *geo = static_cast<const T *>(h->geo16);
    const dim3 fg(static_cast<unsigned>(nitem)), fb(kFvThreads);
    const size_t sm = FvSmem<T>::bytes;
    launch(h, K_FUSED1, "fused_stage1", [&] {
        k_fused_fv<T, 1, false><<<fg, fb, sm, s>>>(fn, s1, fn, B, C, tau, mac, nullptr, G, W, geo);
    });
    launch(h, K_FUSED2, "fused_stage2", [&] {
        k_fused_fv<T, 2, false><<<fg, fb, sm, s>>>(s1, s0, fn, B, C, tau, mac, nullptr, G, W, geo);
    });
    launch(h, K_FUSED3, "fused_stage3", [&] {
        if (stats)
            k_fused_fv<T, 3, true><<<fg, fb, sm, s>>>(s0, s1, fn, B, C, tau, mac, h->d_partial, G, W, geo);
        else
            k_fused_fv<T, 3, false><<<fg, fb, sm, s>>>(s0, s1, fn, B, C, tau, mac, nullptr, G, W, geo);
    });
}

template <class T>
void enqueue_fused_fv(fvlbm_handle *h, bool stats) {
    cudaStream_t s = h->stream;
    fv_stages<T>(h, stats, 0, h->fv.nitem, s);
    if (stats)
        launch(h, K_REDUCE, "reduce", [&] {
            k_reduce_instances<<<h->ninst, kTile, 0, s>>>(h->d_partial, h->fv.d_inst_item0, h->d_inst_sums);
        });
}

// Gradient of f for the two-pass kernels, with the limiter variant when an instance asks for it.
template <class T>
void grad_f(const fvlbm_handle *h, dim3 grid, dim3 block, cudaStream_t s, const T *f, T *g,
            const Geo<T> &G) {
    if (h->limit_f)
        k_grad<T, true><<<grid, block, 0, s>>>(f, g, G);
    else
        k_grad<T, false><<<grid, block, 0, s>>>(f, g, G);
}

// One launch of an SST kernel per contiguous run of SST tiles: f(blocks, first tile).
template <class F>
void for_sst_runs(const fvlbm_handle *h, F &&f) {
    for (const int2 &r : h->sst_runs) f(dim3(static_cast<unsigned>(r.y)), r.x);
}

// The two SST kernels of the two-pass path (unpacked gradients, geometry read as stored), on
// stream h->stream: gradients and f1 of the macros mac, then k, omega, nu_t and tau_out.
template <class T>
void sst_grad_twopass(const fvlbm_handle *h, const T *mac, const T *kc, const T *wc, T *sg, T *f1,
                      const Geo<T> &G, const CompactGeo<T> &CG) {
    for_sst_runs(h, [&](dim3 g, int t0) {
        k_sst_grad<T, false><<<g, kTile, 0, h->stream>>>(mac, kc, wc, sg, f1, G, CG, nullptr, nullptr,
                                                         nullptr, false, t0);
    });
}
template <class T>
void sst_update_twopass(const fvlbm_handle *h, const T *mac, const T *kc, const T *wc, const T *nc,
                        const T *sg, const T *f1, T *kn, T *wn, T *nn, T *tau_out, const Geo<T> &G,
                        const CompactGeo<T> &CG) {
    for_sst_runs(h, [&](dim3 g, int t0) {
        if (h->nonorth)
            k_sst_update<T, false, true><<<g, kTile, 0, h->stream>>>(mac, kc, wc, nc, sg, f1, kn, wn, nn, tau_out,
                                                                     G, nullptr, nullptr, CG, nullptr, nullptr, t0);
        else
            k_sst_update<T, false, false><<<g, kTile, 0, h->stream>>>(mac, kc, wc, nc, sg, f1, kn, wn, nn, tau_out,
                                                                      G, nullptr, nullptr, CG, nullptr, nullptr, t0);
    });
}

template <class T>
void enqueue_step(fvlbm_handle *h, bool stats) {
    Geo<T> G = geo_of<T>(h);
    const dim3 grid(h->ntiles), block(kTile);
    cudaStream_t s = h->stream;
    T *fn = static_cast<T *>(h->fn), *s0 = static_cast<T *>(h->s0), *s1 = static_cast<T *>(h->s1);
    T *B = static_cast<T *>(h->bacc), *C = static_cast<T *>(h->cacc);
    T *g = static_cast<T *>(h->grad), *tau = static_cast<T *>(h->tau), *mac = static_cast<T *>(h->mac);
    if (h->sst) {
        const int c = h->turb, n = 1 - h->turb;
        T *kc = static_cast<T *>(h->kk[c]), *wc = static_cast<T *>(h->ww[c]);
        T *nc = static_cast<T *>(h->nut[c]);
        T *kn = static_cast<T *>(h->kk[n]), *wn = static_cast<T *>(h->ww[n]);
        T *nn = static_cast<T *>(h->nut[n]);
        T *sg = static_cast<T *>(h->sgrad), *f1 = static_cast<T *>(h->f1);
        const CompactGeo<T> CG{static_cast<const T *>(h->gq), static_cast<const T *>(h->dvec)};
        if constexpr (kHasFused<T>) {
            if (h->config != 2) {  // compact geometry, and stage 1's f^(1) with the new tau
                T *r8 = static_cast<T *>(h->sst_rec8), *r2 = static_cast<T *>(h->sst_rec2);
                launch(h, K_SST_GRAD, "sst_grad", [&] {
                    for_sst_runs(h, [&](dim3 sg_grid, int t0) {
                        k_sst_grad<T, true><<<sg_grid, block, 0, s>>>(mac, kc, wc, sg, f1, G, CG, nc, r8, r2,
                                                                      !h->nonorth, t0);
                    });
                });
                launch(h, K_SST_UPDATE, "sst_update", [&] {
                    // the face-value stages relax f^n themselves; the other fused form reads
                    // stage 1's f^(1), relaxed here with the new tau
                    T *fr = h->config == 3 ? nullptr : static_cast<T *>(h->frel);
                    for_sst_runs(h, [&](dim3 sg_grid, int t0) {
                        if (h->nonorth)
                            k_sst_update<T, true, true><<<sg_grid, block, 0, s>>>(
                                mac, kc, wc, nc, sg, f1, kn, wn, nn, tau, G, fn, fr, CG, r8, r2, t0);
                        else
                            k_sst_update<T, true, false><<<sg_grid, block, 0, s>>>(
                                mac, kc, wc, nc, sg, f1, kn, wn, nn, tau, G, fn, fr, CG, r8, r2, t0);
                    });
                });
            }
        }
        if (h->config == 2) {
            launch(h, K_SST_GRAD, "sst_grad", [&] { sst_grad_twopass<T>(h, mac, kc, wc, sg, f1, G, CG); });
            launch(h, K_SST_UPDATE, "sst_update", [&] {
                sst_update_twopass<T>(h, mac, kc, wc, nc, sg, f1, kn, wn, nn, tau, G, CG);
            });
        }
        if (h->per_stage && h->scheme == 0) {
            // per-stage SST reading (two-pass kernels): the SST is solved again from t^n before
            // stages 2 and 3 with the macros of f^(1) and f^(2); stage J relaxes with tau^(J)
            T *t1 = static_cast<T *>(h->tau1), *m2 = static_cast<T *>(h->mac2);
            auto solve = [&](T *macp, T *tau_out) {
                launch(h, K_SST_GRAD, "sst_grad", [&] { sst_grad_twopass<T>(h, macp, kc, wc, sg, f1, G, CG); });
                launch(h, K_SST_UPDATE, "sst_update", [&] {
                    sst_update_twopass<T>(h, macp, kc, wc, nc, sg, f1, kn, wn, nn, tau_out, G, CG);
                });
            };
            // the solve of the step start already ran above into tau; stage 1 relaxes with it
            launch(h, K_STAGE1, "stage1", [&] { k_stage1<T><<<grid, block, 0, s>>>(fn, s0, tau, G); });
            cudaMemcpyAsync(t1, tau, sizeof(T) * static_cast<size_t>(h->np), cudaMemcpyDeviceToDevice, s);
            launch(h, K_MACROS, "stage_macros", [&] { k_stage_macros<T><<<grid, block, 0, s>>>(s0, m2, G); });
            solve(m2, tau);
            launch(h, K_GRAD, "grad_f", [&] { grad_f<T>(h, grid, block, s, s0, g, G); });
            launch(h, K_FLUX1, "flux_stage1", [&] {
                k_flux_stage<T, 1, false><<<grid, block, 0, s>>>(s0, g, s1, fn, B, C, tau, mac, nullptr, G, t1);
            });
            launch(h, K_MACROS, "stage_macros", [&] { k_stage_macros<T><<<grid, block, 0, s>>>(s1, m2, G); });
            solve(m2, tau);
            launch(h, K_GRAD, "grad_f", [&] { grad_f<T>(h, grid, block, s, s1, g, G); });
            launch(h, K_FLUX2, "flux_stage2", [&] {
                k_flux_stage<T, 2, false><<<grid, block, 0, s>>>(s1, g, s0, fn, B, C, tau, mac, nullptr, G);
            });
            launch(h, K_GRAD, "grad_f", [&] { grad_f<T>(h, grid, block, s, s0, g, G); });
            if (stats) {
                launch(h, K_FLUX3, "flux_stage3", [&] {
                    k_flux_stage<T, 3, true><<<grid, block, 0, s>>>(s0, g, s1, fn, B, C, tau, mac, h->d_partial, G);
                });
                launch(h, K_REDUCE, "reduce", [&] {
                    k_reduce_instances<<<h->ninst, kTile, 0, s>>>(h->d_partial, h->d_inst_tile0, h->d_inst_sums);
                });
            } else {
                launch(h, K_FLUX3, "flux_stage3", [&] {
                    k_flux_stage<T, 3, false><<<grid, block, 0, s>>>(s0, g, s1, fn, B, C, tau, mac, nullptr, G);
                });
            }
            h->turb = n;
            return;
        }
        h->turb = n;
    }
    if (h->scheme == 1) {  // explicit Euler: gradient, flux + collision into s0, copy back
        launch(h, K_GRAD, "grad_f", [&] { grad_f<T>(h, grid, block, s, fn, g, G); });
        if (stats) {
            launch(h, K_EULER, "euler", [&] {
                k_flux_stage<T, 4, true><<<grid, block, 0, s>>>(fn, g, s0, fn, B, C, tau, mac, h->d_partial, G);
            });
            launch(h, K_REDUCE, "reduce", [&] {
                k_reduce_instances<<<h->ninst, kTile, 0, s>>>(h->d_partial, h->d_inst_tile0, h->d_inst_sums);
            });
        } else {
            launch(h, K_EULER, "euler", [&] {
                k_flux_stage<T, 4, false><<<grid, block, 0, s>>>(fn, g, s0, fn, B, C, tau, mac, nullptr, G);
            });
        }
        cudaMemcpyAsync(fn, s0, sizeof(T) * kQ * static_cast<size_t>(h->np), cudaMemcpyDeviceToDevice, s);
        return;
    }
    if constexpr (kHasFused<T>) {
        if (h->config == 3) {
            enqueue_fused_fv<T>(h, stats);
            return;
        }
        if (h->config == 0) {
            enqueue_fused<T, 256>(h, stats, h->hs[0]);
            return;
        }
        if (h->config == 1) {
            enqueue_fused<T, 128>(h, stats, h->hs[1]);
            return;
        }
    }
    launch(h, K_STAGE1, "stage1", [&] { k_stage1<T><<<grid, block, 0, s>>>(fn, s0, tau, G); });
    launch(h, K_GRAD, "grad_f", [&] { grad_f<T>(h, grid, block, s, s0, g, G); });
    launch(h, K_FLUX1, "flux_stage1", [&] {
        k_flux_stage<T, 1, false><<<grid, block, 0, s>>>(s0, g, s1, fn, B, C, tau, mac, nullptr, G);
    });
    launch(h, K_GRAD, "grad_f", [&] { grad_f<T>(h, grid, block, s, s1, g, G); });
    launch(h, K_FLUX2, "flux_stage2", [&] {
        k_flux_stage<T, 2, false><<<grid, block, 0, s>>>(s1, g, s0, fn, B, C, tau, mac, nullptr, G);
    });
    launch(h, K_GRAD, "grad_f", [&] { grad_f<T>(h, grid, block, s, s0, g, G); });
    if (stats) {
        launch(h, K_FLUX3, "flux_stage3", [&] {
            k_flux_stage<T, 3, true><<<grid, block, 0, s>>>(s0, g, s1, fn, B, C, tau, mac, h->d_partial, G);
        });
        launch(h, K_REDUCE, "reduce", [&] {
            k_reduce_instances<<<h->ninst, kTile, 0, s>>>(h->d_partial, h->d_inst_tile0, h->d_inst_sums);
        });
    } else {
        launch(h, K_FLUX3, "flux_stage3", [&] {
            k_flux_stage<T, 3, false><<<grid, block, 0, s>>>(s0, g, s1, fn, B, C, tau, mac, nullptr, G);
        });
    }
}

void enqueue(fvlbm_handle *h, bool stats) {
    dispatch(h->precision, [&](auto z_) {
        using T = decltype(z_);
        enqueue_step<T>(h, stats);
    });
}

int launches_per_step(const fvlbm_handle *h) {
    if (h->sst && h->per_stage && h->scheme == 0) return 2 + 1 + 3 + 2 + 3 + 2 + 2;
    return (h->sst ? 2 : 0) + (h->scheme == 1 ? 2 : (h->config != 2 ? 3 : 7));
}

// Capture `nsteps` plain steps into an executable graph.  A replay always starts from the
// k / omega / nu_t ping-pong parity the graph was captured with, and an even step count ends
// on the same parity, so SST runs keep one graph per starting parity.
int build_graph(fvlbm_handle *h, int nsteps, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    const int turb0 = h->turb;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < nsteps; ++k) enqueue(h, false);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    h->turb = turb0;
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e);
    return FVLBM_OK;
}

// Per block of blk cells: ring-1 and ring-2 halo lists and the local adjacency of block and
// ring-1 cells.  The set is marked unusable (ok = false) when a block's halo does not fit the
// 16-bit local index or the shared-memory budget; the two-pass kernels then serve.
template <class T>
int build_halos(fvlbm_handle *h, fvlbm_handle::HaloSet &S, int blk, const std::vector<int> &nbr,
                const std::vector<int> &back, const std::vector<int> &nface,
                const std::vector<int> &inst_tile0) {
    const size_t np = h->np;
    S.blk = blk;
    S.nblk = static_cast<int>(np / blk);
    std::vector<int> local(np, -1), halo_ptr(1, 0), halo, r1n, adj_ptr(1, 0);
    std::vector<unsigned> adj;
    int emax = 0, gmax = 0;
    std::vector<int> ring1, ring2;
    for (int b = 0; b < S.nblk; ++b) {
        const int base = b * blk;
        for (int c = 0; c < blk; ++c) local[base + c] = c;
        ring1.clear();
        ring2.clear();
        int next = blk;
        for (int c = 0; c < blk; ++c)
            for (int m = 0; m < 4; ++m) {
                const int v = nbr[m * np + base + c];
                if (v >= 0 && local[v] < 0) { local[v] = next++; ring1.push_back(v); }
            }
        for (int g : ring1)
            for (int m = 0; m < 4; ++m) {
                const int v = nbr[m * np + g];
                if (v >= 0 && local[v] < 0) { local[v] = next++; ring2.push_back(v); }
            }
        const int E = next, NG = blk + static_cast<int>(ring1.size());
        emax = std::max(emax, E);
        gmax = std::max(gmax, NG);
        halo.insert(halo.end(), ring1.begin(), ring1.end());
        halo.insert(halo.end(), ring2.begin(), ring2.end());
        halo_ptr.push_back(static_cast<int>(halo.size()));
        r1n.push_back(static_cast<int>(ring1.size()));
        const size_t a0 = adj.size();
        adj.resize(a0 + 4 * static_cast<size_t>(NG), kAdjNone);
        for (int c = 0; c < NG; ++c) {
            const int g = c < blk ? base + c : ring1[c - blk];
            for (int m = 0; m < 4; ++m) {
                const int v = nbr[m * np + g];
                unsigned w = kAdjNone;
                if (v == kNone) {
                    w = kAdjNone;
                } else if (v < 0) {
                    w = kAdjBnd | static_cast<unsigned>(-v - 1);
                } else {
                    w = static_cast<unsigned>(local[v]) | (static_cast<unsigned>(back[m * np + g]) << 16) |
                        (nface[v] == 3 ? (1u << 18) : 0u);
                }
                adj[a0 + static_cast<size_t>(m) * NG + c] = w;
            }
        }
        adj_ptr.push_back(adj_ptr.back() + NG);
        for (int c = 0; c < blk; ++c) local[base + c] = -1;
        for (int g : ring1) local[g] = -1;
        for (int g : ring2) local[g] = -1;
    }
    emax = (emax + 3) / 4 * 4;  // 16-byte aligned shared-memory rows
    gmax = (gmax + 3) / 4 * 4;
    const size_t smem = FusedSmem<T>::bytes(emax, gmax);
    if (emax >= 65536 || smem > static_cast<size_t>(kFusedSmemCap)) return FVLBM_OK;  // not usable
    S.emax = emax;
    S.gmax = gmax;
    S.smem = smem;
    int rc;
    std::vector<int> inst_blk0(inst_tile0.size());
    for (size_t q = 0; q < inst_tile0.size(); ++q) inst_blk0[q] = inst_tile0[q] / (blk / kTile);
    if ((rc = upload_raw(h, &S.d_inst_blk0, inst_blk0))) return rc;
    if ((rc = upload_raw(h, &S.d_halo_ptr, halo_ptr))) return rc;
    if (halo.empty()) halo.push_back(0);
    if ((rc = upload_raw(h, &S.d_halo, halo))) return rc;
    if ((rc = upload_raw(h, &S.d_r1, r1n))) return rc;
    if ((rc = upload_raw(h, &S.d_adj_ptr, adj_ptr))) return rc;
    if ((rc = upload_raw(h, &S.d_adj, adj))) return rc;
    // The attribute is per function and process-wide, shared by every handle: always raise it
    // to the library's cap so that a handle with a smaller halo never lowers another's limit.
    const int cap = kFusedSmemCap;
    if (blk == 256) {
        CK(cudaFuncSetAttribute(k_fused_stage<T, 1, false, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
        CK(cudaFuncSetAttribute(k_fused_stage<T, 2, false, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
        CK(cudaFuncSetAttribute(k_fused_stage<T, 3, false, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
        CK(cudaFuncSetAttribute(k_fused_stage<T, 3, true, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    } else {
        CK(cudaFuncSetAttribute(k_fused_stage<T, 1, false, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
        CK(cudaFuncSetAttribute(k_fused_stage<T, 2, false, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
        CK(cudaFuncSetAttribute(k_fused_stage<T, 3, false, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
        CK(cudaFuncSetAttribute(k_fused_stage<T, 3, true, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    }
    S.ok = true;
    return FVLBM_OK;
}

// Work items of the face-value kernel: every 256-cell block whose ring-1 + ring-2 halo and
// ring-1 count fit its shared memory (kFvEcap, kFvGcap) is one item; a block that does not fit
// is split into halves, and a half that does not fit into quarters.  Per item: the ring lists,
// the adjacency words (cell-major) of item and ring-1 cells, and per face which member of each
// direction pair leaves the cell through it -- decided once per face from the FP64 normal of
// one side (e_alpha . n >= 0, the upwind rule of Eq. (advection)) and complemented on the
// other side, so that both sides always agree.  The ring lists and the adjacency sit at fixed
// strides per item (FvItems).  The set is left unusable (ok = false) if a quarter block still
// does not fit.
template <class T>
int build_fv_items(fvlbm_handle *h, const std::vector<int> &nbr, const std::vector<int> &back,
                   const std::vector<double> &sn, const std::vector<int> &inst_tile0) {
    const size_t np = h->np;
    // outgoing bits of every (cell, face slot)
    std::vector<unsigned char> pbits(4 * np, 0);
    for (size_t g = 0; g < np; ++g)
        for (int m = 0; m < 4; ++m) {
            const int v = nbr[m * np + g];
            if (v < 0) continue;
            const int b = back[m * np + g];
            const bool owner = static_cast<size_t>(v) > g || (static_cast<size_t>(v) == g && b > m);
            const size_t cg = owner ? g : static_cast<size_t>(v);
            const int mg = owner ? m : b;
            const double nx = sn[(2 * mg) * np + cg], ny = sn[(2 * mg + 1) * np + cg];
            unsigned bits = 0;
            for (int p = 0; p < 4; ++p) {
                const double en = p == 0 ? nx : (p == 1 ? ny : (p == 2 ? nx + ny : ny - nx));
                if (en >= 0.0) bits |= 1u << p;
            }
            pbits[m * np + g] = static_cast<unsigned char>(owner ? bits : (~bits & 15u));
        }
    std::vector<int4> hdr;
    std::vector<int> halo, ovf, item_inst;
    std::vector<uint4> adj;
    std::vector<int> local(np, -1), ring1, ring2;
    int n_split = 0, n_ovf = 0;
    bool fits_all = true;
    // try one item of cnt cells at base (instance inst); returns false if it does not fit
    auto try_item = [&](int base, int cnt, int inst, bool commit) -> bool {
        for (int c = 0; c < cnt; ++c) local[base + c] = c;
        ring1.clear();
        ring2.clear();
        int next = cnt;
        for (int c = 0; c < cnt; ++c)
            for (int m = 0; m < 4; ++m) {
                const int v = nbr[m * np + base + c];
                if (v >= 0 && local[v] < 0) { local[v] = next++; ring1.push_back(v); }
            }
        for (int g : ring1)
            for (int m = 0; m < 4; ++m) {
                const int v = nbr[m * np + g];
                if (v >= 0 && local[v] < 0) { local[v] = next++; ring2.push_back(v); }
            }
        const int E = next, NG = cnt + static_cast<int>(ring1.size());
        const bool fit = E <= kFvEcap && NG <= kFvGcap && E - cnt <= 2 * kFvHs;
        if (fit && commit) {
            // halo ids: kFvHs slots per item, the rest (split items only: E <= kFvEcap and
            // cnt >= 64 leave at most 2 kFvHs) in a kFvHs-slot chunk of the overflow table
            const int nh = E - cnt;
            const size_t h0 = halo.size();
            halo.resize(h0 + kFvHs, -1);
            int ovf0 = -1;
            if (nh > kFvHs) {
                ++n_ovf;
                ovf0 = static_cast<int>(ovf.size());
                ovf.resize(ovf.size() + kFvHs, -1);
            }
            for (int r = 0; r < nh; ++r) {
                const int g = r < static_cast<int>(ring1.size()) ? ring1[r] : ring2[r - ring1.size()];
                if (r < kFvHs)
                    halo[h0 + r] = g;
                else
                    ovf[ovf0 + r - kFvHs] = g;
            }
            hdr.push_back(make_int4(base, cnt | (static_cast<int>(ring1.size()) << 16), inst, ovf0));
            const size_t a0 = adj.size();
            adj.resize(a0 + kFvGcap, make_uint4(kFvNone, kFvNone, kFvNone, kFvNone));
            for (int c = 0; c < NG; ++c) {
                const int g = c < cnt ? base + c : ring1[c - cnt];
                unsigned w[4];
                for (int m = 0; m < 4; ++m) {
                    const int v = nbr[m * np + g];
                    if (v == kNone)
                        w[m] = kFvNone;
                    else if (v < 0)
                        w[m] = kFvBnd | static_cast<unsigned>(-v - 1);
                    else
                        w[m] = static_cast<unsigned>(local[v]) | (static_cast<unsigned>(back[m * np + g]) << 16) |
                               (static_cast<unsigned>(pbits[m * np + g]) << 18);
                }
                adj[a0 + c] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        for (int c = 0; c < cnt; ++c) local[base + c] = -1;
        for (int g : ring1) local[g] = -1;
        for (int g : ring2) local[g] = -1;
        return fit;
    };
    std::vector<int> tile_inst_of(np / kTile);
    for (size_t q = 0; q + 1 < inst_tile0.size(); ++q)
        for (int tt = inst_tile0[q]; tt < inst_tile0[q + 1]; ++tt) tile_inst_of[tt] = static_cast<int>(q);
    constexpr int IT = kFvThreads, HALF = IT / 2, QUART = IT / 4;
    const int nblk = static_cast<int>(np / IT);
    for (int b = 0; b < nblk && fits_all; ++b) {
        const int base = b * IT;
        int inst = tile_inst_of[base / kTile];
        if (try_item(base, IT, inst, true)) {
            item_inst.push_back(inst);
            continue;
        }
        ++n_split;
        for (int half = 0; half < 2 && fits_all; ++half) {
            const int hb = base + HALF * half;
            if (try_item(hb, HALF, inst, true)) {
                item_inst.push_back(inst);
                continue;
            }
            for (int qq = 0; qq < 2 && fits_all; ++qq) {
                if (try_item(hb + QUART * qq, QUART, inst, true))
                    item_inst.push_back(inst);
                else
                    fits_all = false;
            }
        }
    }
    if (!fits_all || hdr.empty() || ovf.size() >= (1u << 31)) return FVLBM_OK;  // not usable
    const int nitem = static_cast<int>(hdr.size());
    std::vector<int> inst_item0(h->ninst + 1, nitem);
    for (int k = nitem - 1; k >= 0; --k) inst_item0[item_inst[k]] = k;
    for (int q = h->ninst - 1; q >= 0; --q)  // instances without items (none in practice)
        if (inst_item0[q] > inst_item0[q + 1]) inst_item0[q] = inst_item0[q + 1];
    if (ovf.empty()) ovf.push_back(-1);
    int rc;
    if ((rc = upload_raw(h, &h->fv.d_hdr, hdr))) return rc;
    if ((rc = upload_raw(h, &h->fv.d_halo, halo))) return rc;
    if ((rc = upload_raw(h, &h->fv.d_ovf, ovf))) return rc;
    if ((rc = upload_raw(h, &h->fv.d_adj, adj))) return rc;
    if ((rc = upload_raw(h, &h->fv.d_inst_item0, inst_item0))) return rc;
    CK(cudaFuncSetAttribute(k_fused_fv<T, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            static_cast<int>(FvSmem<T>::bytes)));
    CK(cudaFuncSetAttribute(k_fused_fv<T, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            static_cast<int>(FvSmem<T>::bytes)));
    CK(cudaFuncSetAttribute(k_fused_fv<T, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            static_cast<int>(FvSmem<T>::bytes)));
    CK(cudaFuncSetAttribute(k_fused_fv<T, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            static_cast<int>(FvSmem<T>::bytes)));
    h->fv.nitem = nitem;
    h->fv.n_split = n_split;
    h->fv.n_ovf = n_ovf;
    h->fv.ok = true;
    return FVLBM_OK;
}

// f^(1) of the coming step from the current f^n and tau, for every cell (after create and
// set_f); the fused stage-1 kernel reads it.
template <class T>
void relax_all(fvlbm_handle *h) {
    k_stage1<T><<<h->ntiles, kTile, 0, h->stream>>>(static_cast<const T *>(h->fn),
                                                   static_cast<T *>(h->frel),
                                                   static_cast<const T *>(h->tau), geo_of<T>(h));
}

template <class T>
int allocate_state(fvlbm_handle *h, const std::vector<const Prepared *> &P,
                   const std::vector<int> &inst_tile0) {
    const size_t np = h->np;
    int rc;
    const size_t ts = sizeof(T);
    for (void **p : {&h->fn, &h->s0, &h->s1, &h->bacc, &h->cacc, &h->frel})
        if ((rc = dalloc(h, p, kQ * np * ts))) return rc;
    if ((rc = dalloc(h, &h->grad, 2 * kQ * np * ts))) return rc;
    if ((rc = dalloc(h, &h->tau, np * ts))) return rc;
    if ((rc = dalloc(h, &h->mac, 3 * np * ts))) return rc;
    for (int b = 0; b < 2; ++b)
        for (void **p : {&h->kk[b], &h->ww[b], &h->nut[b]})
            if ((rc = dalloc(h, p, np * ts))) return rc;
    if (h->sst && h->per_stage) {
        if ((rc = dalloc(h, &h->tau1, np * ts))) return rc;
        if ((rc = dalloc(h, &h->mac2, 3 * np * ts))) return rc;
    }
    if (h->sst) {
        if ((rc = dalloc(h, &h->sgrad, 12 * np * ts))) return rc;
        if ((rc = dalloc(h, &h->sst_rec8, 8 * np * ts))) return rc;
        if ((rc = dalloc(h, &h->sst_rec2, 2 * np * ts))) return rc;
        if ((rc = dalloc(h, &h->f1, np * ts))) return rc;
    }
    // geometry, concatenated over instances with neighbour / boundary ids offset
    std::vector<int> nbr(4 * np, kNone), back(4 * np, -1), nface(np, 0);
    std::vector<int> btype(h->nbt), bowner(h->nbt), perm;
    std::vector<double> gq(8 * np, 0), dvec(8 * np, 0);
    std::vector<double> sn(8 * np, 0), lsq(8 * np, 0), rown(8 * np, 0), rnbr(8 * np, 0);
    std::vector<double> dinv(4 * np, 0), area(np, 0), wdist(np, 1e30);
    std::vector<double> bval(5 * static_cast<size_t>(h->nbt)), bnrm(2 * static_cast<size_t>(h->nbt));
    std::vector<double> blen(h->nbt);
    std::vector<double> r0(np), u0(np), v0(np), k0(np), w0(np), tau0(np), nut0(np);
    for (int q = 0; q < h->ninst; ++q) {
        const Prepared &p = *P[q];
        const InstInfo &I = h->inst[q];
        const size_t o = I.cell_off, pn = p.np;
        for (int m = 0; m < 4; ++m)
            for (size_t k = 0; k < pn; ++k) {
                const int v = p.nbr[m * pn + k];
                nbr[m * np + o + k] = v == kNone ? kNone : (v >= 0 ? v + I.cell_off : v - I.bface_off);
                back[m * np + o + k] = p.back[m * pn + k];
                dinv[m * np + o + k] = p.dinv[m * pn + k];
            }
        for (int c = 0; c < 8; ++c)
            for (size_t k = 0; k < pn; ++k) {
                sn[c * np + o + k] = p.sn[c * pn + k];
                lsq[c * np + o + k] = p.lsq[c * pn + k];
                rown[c * np + o + k] = p.rown[c * pn + k];
                rnbr[c * np + o + k] = p.rnbr[c * pn + k];
                gq[c * np + o + k] = p.gq[c * pn + k];
                dvec[c * np + o + k] = p.dvec[c * pn + k];
            }
        for (size_t k = 0; k < pn; ++k) nface[o + k] = p.nface[k];
        for (size_t k = 0; k < pn; ++k) {
            area[o + k] = p.area[k];
            wdist[o + k] = p.wdist[k];
            r0[o + k] = p.rho_i[k];
            u0[o + k] = p.u_i[k];
            v0[o + k] = p.v_i[k];
            k0[o + k] = p.k_i[k];
            w0[o + k] = p.w_i[k];
            nut0[o + k] = I.sst ? p.k_i[k] / p.w_i[k] : 0.0;
            tau0[o + k] = (I.nu + nut0[o + k]) / kCs2;
        }
        for (int b = 0; b < p.nb; ++b) {
            const int gb = I.bface_off + b;
            btype[gb] = p.btype[b];
            bowner[gb] = p.bowner[b] + I.cell_off;
            for (int c = 0; c < 5; ++c) bval[c * h->nbt + gb] = p.bval[5 * b + c];
            bnrm[gb] = p.bnrm[2 * b];
            bnrm[h->nbt + gb] = p.bnrm[2 * b + 1];
            blen[gb] = p.blen[b];
        }
        for (int k = 0; k < p.nc; ++k) perm.push_back(p.perm[k]);
    }
    if ((rc = upload_raw(h, &h->d_nbr, nbr))) return rc;
    if ((rc = upload_raw(h, &h->d_btype, btype))) return rc;
    if ((rc = upload_raw(h, &h->d_bowner, bowner))) return rc;
    if ((rc = upload_raw(h, &h->d_perm, perm))) return rc;
    {  // FNV-1a over the internal order of every instance (state blobs check it)
        unsigned long long hsh = 1469598103934665603ull;
        for (int q = 0; q < h->ninst; ++q) {
            hsh = (hsh ^ static_cast<unsigned long long>(P[q]->np)) * 1099511628211ull;
            for (int v : P[q]->perm) hsh = (hsh ^ static_cast<unsigned long long>(v)) * 1099511628211ull;
        }
        h->order_hash = hsh;
    }
    {
        std::vector<int> map, inv(h->np, -1);
        int out_off = 0;
        for (int q = 0; q < h->ninst; ++q) {
            const Prepared &p = *P[q];
            map.resize(out_off + p.nc);
            for (int k = 0; k < p.nc; ++k) {
                map[out_off + p.perm[k]] = h->inst[q].cell_off + k;
                inv[h->inst[q].cell_off + k] = out_off + p.perm[k];
            }
            out_off += p.nc;
        }
        h->total_nc = out_off;
        if ((rc = upload_raw(h, &h->d_all_map, map))) return rc;
        if ((rc = upload_raw(h, &h->d_all_inv, inv))) return rc;
    }
    if ((rc = upload_as<T>(h, &h->sn, sn))) return rc;
    if ((rc = upload_as<T>(h, &h->lsq, lsq))) return rc;
    if ((rc = upload_as<T>(h, &h->rown, rown))) return rc;
    if ((rc = upload_as<T>(h, &h->rnbr, rnbr))) return rc;
    if ((rc = upload_as<T>(h, &h->dinv, dinv))) return rc;
    if ((rc = upload_as<T>(h, &h->area, area))) return rc;
    if ((rc = upload_as<T>(h, &h->wdist, wdist))) return rc;
    if ((rc = upload_as<T>(h, &h->bval, bval))) return rc;
    if ((rc = upload_as<T>(h, &h->bnrm, bnrm))) return rc;
    if ((rc = upload_as<T>(h, &h->blen, blen))) return rc;
    if (std::is_same<T, double>::value)
        if ((rc = upload_raw(h, &h->d_back, back))) return rc;
    bool any_local = false;
    for (const Prepared *p : P) any_local |= !p->dt_cell.empty();
    if (any_local) {  // local time stepping: every cell's step (global instances: their dt)
        std::vector<double> dtc(np, 1.0);
        for (int q = 0; q < h->ninst; ++q) {
            const Prepared &p = *P[q];
            for (int k = 0; k < p.np; ++k)
                dtc[h->inst[q].cell_off + k] = p.dt_cell.empty() ? p.dt : p.dt_cell[k];
        }
        if ((rc = upload_as<T>(h, &h->dtc, dtc))) return rc;
    }
    if (h->fused) {
        if ((rc = upload_as<T>(h, &h->gq, gq))) return rc;
        if ((rc = upload_raw(h, &h->d_err, std::vector<int>(1, 0)))) return rc;
        if ((rc = upload_as<T>(h, &h->dvec, dvec))) return rc;
    }
    if constexpr (kHasFused<T>) {
        if (h->fused) {
            if ((rc = build_halos<T>(h, h->hs[0], 256, nbr, back, nface, inst_tile0))) return rc;
            if ((rc = build_halos<T>(h, h->hs[1], 128, nbr, back, nface, inst_tile0))) return rc;
            if ((rc = build_fv_items<T>(h, nbr, back, sn, inst_tile0))) return rc;
            if (h->fv.ok) {  // cell-major geometry of the face-value kernels (64 B per cell)
                std::vector<double> g16(16 * np);
                for (size_t k = 0; k < np; ++k)
                    for (int c = 0; c < 8; ++c) {
                        g16[16 * k + c] = gq[c * np + k];
                        g16[16 * k + 8 + c] = lsq[c * np + k];
                    }
                if ((rc = upload_as<T>(h, &h->geo16, g16))) return rc;
            }
            h->config = h->hs[0].ok ? 0 : (h->hs[1].ok ? 1 : 2);
            if (h->fv.ok && (h->kernel_path == 2 || h->config == 2)) h->config = 3;
            // FP32: only the forms whose least-squares weights come from the host in FP64 (the
            // 256- and 128-cell forms invert M on chip, in FP32 a few digits on y+ ~ 1 cells)
            if (h->precision == FVLBM_FP32_DEV) h->config = h->fv.ok ? 3 : 2;
            if (h->config == 2) h->fused = false;
        }
    }
    {
        std::vector<double> kt(k0), wt(w0);
        void *tmp = nullptr;
        for (int b = 0; b < 2; ++b) {
            std::vector<T> a(kt.begin(), kt.end()), c(wt.begin(), wt.end()), n(nut0.begin(), nut0.end());
            CK(cudaMemcpy(h->kk[b], a.data(), np * ts, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(h->ww[b], c.data(), np * ts, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(h->nut[b], n.data(), np * ts, cudaMemcpyHostToDevice));
        }
        (void)tmp;
        std::vector<T> t(tau0.begin(), tau0.end());
        CK(cudaMemcpy(h->tau, t.data(), np * ts, cudaMemcpyHostToDevice));
    }
    // initial state: f = f^eq(rho, u) (Step 0)
    double *d_init = nullptr;
    if ((rc = dalloc(h, reinterpret_cast<void **>(&d_init), 3 * np * sizeof(double)))) return rc;
    CK(cudaMemcpy(d_init, r0.data(), np * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_init + np, u0.data(), np * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_init + 2 * np, v0.data(), np * sizeof(double), cudaMemcpyHostToDevice));
    Geo<T> G = geo_of<T>(h);
    k_init_state<T><<<h->ntiles, kTile, 0, h->stream>>>(static_cast<T *>(h->fn), static_cast<T *>(h->mac),
                                                       d_init, d_init + np, d_init + 2 * np, G);
    CK(cudaGetLastError());
    relax_all<T>(h);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return FVLBM_OK;
}

void free_all(fvlbm_handle *h) {
    auto &A = h->aio;
    if (A.init) {
        cudaStreamSynchronize(A.s_in);
        cudaStreamSynchronize(A.s_out);
        for (int k = 0; k < 2; ++k) {
            if (A.d_in[k]) cudaFree(A.d_in[k]);
            if (A.d_out[k]) cudaFree(A.d_out[k]);
            for (cudaEvent_t e : {A.in_ready[k], A.in_free[k], A.out_ready[k], A.out_free[k]})
                cudaEventDestroy(e);
        }
        cudaStreamDestroy(A.s_in);
        cudaStreamDestroy(A.s_out);
        A.init = false;
    }
    for (int k = 0; k < 3; ++k)
        if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

int create_impl(int n, const fvlbm_mesh *meshes, const fvlbm_bc *bcs, const fvlbm_params *params,
                int device, void *stream, fvlbm_handle **out) {
    if (!out || n <= 0 || !meshes || !bcs || !params) return FVLBM_ERR_BAD_PARAM;
    *out = nullptr;
    const int prec = params[0].precision;
    int sst = 0;
    if (prec != FVLBM_FP64 && prec != FVLBM_FP32_DEV && prec != FVLBM_FP64_TANGENT)
        return FVLBM_ERR_BAD_PARAM;
    for (int q = 0; q < n; ++q) {
        if (params[q].precision != prec || params[q].scheme != params[0].scheme)
            return FVLBM_ERR_BAD_PARAM;
        sst |= params[q].sst ? 1 : 0;
    }
    std::vector<std::unique_ptr<Prepared>> prep(n);
    std::vector<const Prepared *> P(n);
    for (int q = 0; q < n; ++q) {
        prep[q].reset(new Prepared());
        std::string why;
        const int rc = prepare_instance(meshes[q], bcs[q], params[q], prep[q].get(), &why);
        if (rc) {
            fprintf(stderr, "fvlbm_create: instance %d: %s\n", q, why.c_str());
            return rc;
        }
        P[q] = prep[q].get();
    }
    std::unique_ptr<fvlbm_handle> h(new fvlbm_handle());
    if (device < 0) {
        if (cudaGetDevice(&device) != cudaSuccess) return FVLBM_ERR_CUDA;
    }
    h->device = device;
    CK(cudaSetDevice(device));
    h->precision = prec;
    h->sst = sst != 0;
    h->scheme = params[0].scheme;
    if (h->scheme != 0 && h->scheme != 1) return FVLBM_ERR_BAD_PARAM;
    for (int q = 0; q < n; ++q) {
        h->limit_f |= (params[q].variant & 1) != 0;
        h->nonorth |= (params[q].variant & (2 | 8)) != 0;
        if (((params[q].variant ^ params[0].variant) & 4) != 0) return FVLBM_ERR_BAD_PARAM;
    }
    h->per_stage = (params[0].variant & 4) != 0;
    // The fused and compact-geometry kernels derive n dl of a face from the cell's own nodes.
    // Across a periodic pair whose edges agree only to a file's precision, side B's own edge
    // is not side A's reversed, which every other path uses for both sides (one face, one
    // flux): such handles keep the precomputed geometry of the two-pass kernels.
    bool periodic_inexact = false;
    for (int q = 0; q < n; ++q) periodic_inexact |= !(P[q]->periodic_gap <= 1e-12);
    h->kernel_path = params[0].kernel_path;
    if (h->kernel_path < 0 || h->kernel_path > 2) return FVLBM_ERR_BAD_PARAM;
    h->fused = h->kernel_path != 1 && h->scheme == 0 && prec != FVLBM_FP64_TANGENT &&
               !h->limit_f && !h->per_stage && !periodic_inexact;
    h->ninst = n;
    int cell_off = 0, bface_off = 0;
    std::vector<int> tile_inst, inst_tile0;
    std::vector<InstParam> ip(n);
    for (int q = 0; q < n; ++q) {
        const Prepared &p = *P[q];
        InstInfo I;
        I.nc = p.nc;
        I.np = p.np;
        I.nb = p.nb;
        I.n_bedges_in = p.n_bedges_in;
        I.sst = params[q].sst ? 1 : 0;
        I.cell_off = cell_off;
        I.tile_off = cell_off / kTile;
        I.bface_off = bface_off;
        I.dt = p.dt;
        I.rho0 = params[q].rho0;
        I.uref = params[q].uref;
        I.lref = params[q].lref;
        I.alpha_deg = params[q].alpha_deg;
        I.nu = params[q].nu;
        I.bedge_of = p.bedge_of;
        I.n_nodes = meshes[q].n_nodes;
        if (prec == FVLBM_FP64_TANGENT || prec == FVLBM_FP64) {  // shape derivatives need the mesh
            const fvlbm_mesh &M = meshes[q];
            const fvlbm_bc &B = bcs[q];
            auto mc = std::make_shared<MeshCopy>();
            mc->xy.assign(M.xy, M.xy + 2 * static_cast<size_t>(M.n_nodes));
            mc->cell_ptr.assign(M.cell_ptr, M.cell_ptr + M.n_cells + 1);
            mc->cell_nodes.assign(M.cell_nodes, M.cell_nodes + M.cell_ptr[M.n_cells]);
            mc->bnodes.assign(B.bedge_nodes, B.bedge_nodes + 2 * static_cast<size_t>(B.n_bedges));
            mc->btype.assign(B.bedge_type, B.bedge_type + B.n_bedges);
            mc->bval.assign(B.bedge_val, B.bedge_val + 5 * static_cast<size_t>(B.n_bedges));
            if (B.n_periodic > 0) {
                mc->ppairs.assign(B.periodic_pairs, B.periodic_pairs + 2 * static_cast<size_t>(B.n_periodic));
                mc->pshift.assign(B.periodic_shift, B.periodic_shift + 2 * static_cast<size_t>(B.n_periodic));
            }
            mc->perm = p.perm;
            mc->params = params[q];
            mc->params.rho_init = mc->params.u_init = mc->params.v_init = nullptr;
            mc->params.k_init = mc->params.omega_init = nullptr;
            mc->params.dt = p.dt;  // the time step is held fixed under differentiation
            I.mesh = mc;
        }
        inst_tile0.push_back(I.tile_off);
        for (int t = 0; t < p.np / kTile; ++t) tile_inst.push_back(q);
        ip[q] = InstParam{p.dt, params[q].nu, params[q].rho0,
                          1e-12 * params[q].uref / params[q].lref, params[q].sst ? 1 : 0,
                          p.dt_cell.empty() ? 0 : 1, params[q].variant};
        ip[q].dt_f = static_cast<float>(ip[q].dt);
        ip[q].nu_f = static_cast<float>(ip[q].nu);
        ip[q].rho0_f = static_cast<float>(ip[q].rho0);
        ip[q].omega_min_f = static_cast<float>(ip[q].omega_min);
        cell_off += p.np;
        bface_off += p.nb;
        h->inst.push_back(I);
    }
    inst_tile0.push_back(cell_off / kTile);
    for (int q = 0; q < n; ++q) {  // contiguous runs of SST tiles: the SST kernels visit these only
        const int t0 = h->inst[q].tile_off, nt = h->inst[q].np / kTile;
        if (!params[q].sst || nt == 0) continue;
        if (!h->sst_runs.empty() && h->sst_runs.back().x + h->sst_runs.back().y == t0)
            h->sst_runs.back().y += nt;
        else
            h->sst_runs.push_back(make_int2(t0, nt));
    }
    h->np = cell_off;
    h->nbt = bface_off;
    h->ntiles = cell_off / kTile;
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    int rc;
    if ((rc = upload_raw(h.get(), &h->d_tile_inst, tile_inst))) { free_all(h.get()); return rc; }
    if ((rc = upload_raw(h.get(), &h->d_inst_tile0, inst_tile0))) { free_all(h.get()); return rc; }

    if ((rc = upload_raw(h.get(), &h->d_ip, ip))) { free_all(h.get()); return rc; }
    if ((rc = dalloc(h.get(), reinterpret_cast<void **>(&h->d_partial), 4 * sizeof(double) * h->ntiles)) ||
        (rc = dalloc(h.get(), reinterpret_cast<void **>(&h->d_inst_sums), 4 * sizeof(double) * n))) {
        free_all(h.get());
        return rc;
    }
    dispatch(prec, [&](auto z_) { rc = allocate_state<decltype(z_)>(h.get(), P, inst_tile0); });
    if (rc) {
        free_all(h.get());
        return rc;
    }
    *out = h.release();
    return FVLBM_OK;
}

int io_buffer(fvlbm_handle *h, size_t bytes) {
    if (h->io_bytes >= bytes) return FVLBM_OK;
    if (h->d_io) {
        cudaFree(h->d_io);
        h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), static_cast<void *>(h->d_io)));
        h->device_bytes -= h->io_bytes;
        h->d_io = nullptr;
    }
    int rc = dalloc(h, reinterpret_cast<void **>(&h->d_io), bytes);
    if (rc) return rc;
    h->io_bytes = bytes;
    return FVLBM_OK;
}

int perm_offset(const fvlbm_handle *h, int instance) {
    int o = 0;
    for (int q = 0; q < instance; ++q) o += h->inst[q].nc;
    return o;
}

// Cells addressed by an instance argument (FVLBM_ALL_INSTANCES: all of them).
size_t io_cells(const fvlbm_handle *h, int instance) {
    return instance == -1 ? static_cast<size_t>(h->total_nc) : static_cast<size_t>(h->inst[instance].nc);
}

// f^(1) of the coming step is kept only for the 256- and 128-cell fused forms (configurations
// 0, 1); a switch to them (the autotuner) or a load relaxes it again from f^n.
void *frel_target(const fvlbm_handle *h) { return h->config == 0 || h->config == 1 ? h->frel : nullptr; }

// The state from a DEVICE buffer (input cell order, [cells][9]; IN = double: absolute f,
// float: FP32 deviations) into f^n, the macros and f^(1) of the coming step; handle's stream.
template <class IN>
void scatter_state_dev(fvlbm_handle *h, int instance, const IN *src) {
    // the internal cells of the instance (all instances: every cell), padding included
    const int i0 = instance == -1 ? 0 : h->inst[instance].cell_off;
    const int n = instance == -1 ? static_cast<int>(h->np) : h->inst[instance].np;
    const int po = instance == -1 ? 0 : perm_offset(h, instance);
    dispatch(h->precision, [&](auto z_) {
        using T = decltype(z_);
        k_scatter_state<T, IN><<<(n + 255) / 256, 256, 0, h->stream>>>(
            static_cast<T *>(h->fn), static_cast<T *>(h->mac), static_cast<T *>(frel_target(h)),
            static_cast<const T *>(h->tau), h->d_all_inv, i0, n, po, geo_of<T>(h), src);
    });
}

// Selected fields (mask bits: rho, u, v, k, omega, nu_t) into a DEVICE buffer, field-major
// [6][cells] in input cell order.
void gather_fields_dev(fvlbm_handle *h, int instance, unsigned mask, double *dst) {
    const int n = static_cast<int>(io_cells(h, instance));
    const int po = instance == -1 ? 0 : perm_offset(h, instance);
    const int c = h->turb;
    dispatch(h->precision, [&](auto z_) {
        using T = decltype(z_);
        k_gather_fields_map<T><<<(n + 255) / 256, 256, 0, h->stream>>>(
            static_cast<T *>(h->mac), static_cast<T *>(h->kk[c]), static_cast<T *>(h->ww[c]),
            static_cast<T *>(h->nut[c]), h->d_all_map + po, n, h->np, mask, dst);
    });
}

unsigned field_mask(const double *const *dst) {
    unsigned m = 0;
    for (int q = 0; q < 6; ++q)
        if (dst[q]) m |= 1u << q;
    return m;
}

// Pipelined host I/O: two staging slots per direction and two transfer streams, so that
// host-device copies run on the copy engines while the compute stream steps.
int async_init(fvlbm_handle *h) {
    auto &A = h->aio;
    if (A.init) return FVLBM_OK;
    CK(cudaStreamCreateWithFlags(&A.s_in, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&A.s_out, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k)
        for (cudaEvent_t *e : {&A.in_ready[k], &A.in_free[k], &A.out_ready[k], &A.out_free[k]}) {
            CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
            CK(cudaEventRecord(*e, h->stream));
        }
    A.init = true;
    return FVLBM_OK;
}

int async_slot(fvlbm_handle *h, double **buf, size_t *cap, size_t bytes) {
    if (*cap >= bytes) return FVLBM_OK;
    // growing a slot: let everything in flight finish first
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaStreamSynchronize(h->aio.s_in));
    CK(cudaStreamSynchronize(h->aio.s_out));
    if (*buf) CK(cudaFree(*buf));
    *buf = nullptr;
    *cap = 0;
    CK(cudaMalloc(reinterpret_cast<void **>(buf), bytes));
    *cap = bytes;
    return FVLBM_OK;
}

// Wall force and coefficients of one instance; dout (may be NULL) receives their derivatives
// (tangent handles), dalpha the derivative of the free-stream angle in radians; fsrc (may be
// NULL: the current state) the distributions they are taken from.
int forces_impl(fvlbm_handle *h, int instance, double dalpha, double *out, double *dout, double *cp,
                const void *fsrc = nullptr, double *fxy = nullptr) {
    if (!h || instance < 0 || instance >= h->ninst || !out) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    const InstInfo &I = h->inst[instance];
    const int nbi = I.nb;
    int rc = io_buffer(h, sizeof(double) * 5 * std::max(nbi, 1));
    if (rc) return rc;
    if (nbi > 0) {
        const int nb = (nbi + 255) / 256;
        dispatch(h->precision, [&](auto z_) {
            using T = decltype(z_);
            k_wall_forces<T><<<nb, 256, 0, h->stream>>>(
                static_cast<const T *>(fsrc ? fsrc : h->fn), h->d_bowner, static_cast<T *>(h->bnrm),
                static_cast<T *>(h->blen), I.bface_off, nbi, I.rho0, I.uref, geo_of<T>(h), h->d_io);
        });
        CK(cudaGetLastError());
    }
    std::vector<double> host(5 * static_cast<size_t>(std::max(nbi, 1)));
    CK(cudaMemcpyAsync(host.data(), h->d_io, host.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double fx = 0, fy = 0, dfx = 0, dfy = 0;
    if (cp)
        for (int b = 0; b < I.n_bedges_in; ++b) cp[b] = 0.0;
    if (fxy)
        for (int b = 0; b < 2 * I.n_bedges_in; ++b) fxy[b] = 0.0;
    for (int b = 0; b < nbi; ++b) {
        fx += host[b];
        fy += host[nbi + b];
        dfx += host[3 * nbi + b];
        dfy += host[4 * nbi + b];
        if (cp) cp[I.bedge_of[b]] = host[2 * nbi + b];
        if (fxy) {
            fxy[2 * I.bedge_of[b]] = host[b];
            fxy[2 * I.bedge_of[b] + 1] = host[nbi + b];
        }
    }
    const double q = 0.5 * I.rho0 * I.uref * I.uref;
    const double al = I.alpha_deg * M_PI / 180.0;
    out[0] = fx;
    out[1] = fy;
    out[2] = (fx * std::cos(al) + fy * std::sin(al)) / (q * I.lref);
    out[3] = (-fx * std::sin(al) + fy * std::cos(al)) / (q * I.lref);
    if (dout) {
        // C_D = (Fx cos a + Fy sin a) / (q l), C_L = (-Fx sin a + Fy cos a) / (q l)
        const double ca = std::cos(al), sa = std::sin(al);
        dout[0] = dfx;
        dout[1] = dfy;
        dout[2] = (dfx * ca + dfy * sa + dalpha * (-fx * sa + fy * ca)) / (q * I.lref);
        dout[3] = (-dfx * sa + dfy * ca - dalpha * (fx * ca + fy * sa)) / (q * I.lref);
    }
    return FVLBM_OK;
}

}  // namespace

#include "fvlbm_adjoint.cuh"

extern "C" {

int fvlbm_create(const fvlbm_mesh *mesh, const fvlbm_bc *bc, const fvlbm_params *params,
                 int device, void *stream, fvlbm_handle **out) {
    return create_impl(1, mesh, bc, params, device, stream, out);
}

int fvlbm_create_batch(int n, const fvlbm_mesh *meshes, const fvlbm_bc *bcs,
                       const fvlbm_params *params, int device, void *stream, fvlbm_handle **out) {
    return create_impl(n, meshes, bcs, params, device, stream, out);
}

int fvlbm_step(fvlbm_handle *h, int n_steps, fvlbm_stats *stats) {
    if (!h || n_steps < 0) return FVLBM_ERR_BAD_PARAM;
    NvtxScope range("fvlbm_step");
    CK(cudaSetDevice(h->device));
    int remaining = n_steps;
    const bool want_stats = stats != nullptr && n_steps > 0;
    if (want_stats) --remaining;  // the last step runs un-captured with the reductions
    // graphs: laminar runs replay freely; SST runs keep the ping-pong parity (graphs of an
    // even number of steps only)
    while (remaining >= kGraphSteps) {
        const int gi = 1 + (h->sst ? h->turb : 0);
        if (!h->graph[gi]) {
            int rc = build_graph(h, kGraphSteps, &h->graph[gi]);
            if (rc) return rc;
        }
        CK(cudaGraphLaunch(h->graph[gi], h->stream));
        remaining -= kGraphSteps;
        h->steps += kGraphSteps;
    }
    while (remaining > 0) {
        if (!h->sst) {
            if (!h->graph[0]) {
                int rc = build_graph(h, 1, &h->graph[0]);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(h->graph[0], h->stream));
        } else {
            enqueue(h, false);
        }
        --remaining;
        ++h->steps;
    }
    if (want_stats) {
        enqueue(h, true);
        ++h->steps;
    }
    CK(cudaGetLastError());
    if (want_stats) {
        std::vector<double> sums(4 * static_cast<size_t>(h->ninst));
        CK(cudaMemcpyAsync(sums.data(), h->d_inst_sums, sums.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
        int err = 0;
        if (h->d_err)
            CK(cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (err) {
            fprintf(stderr, "fvlbm_step: a fused-kernel staging wait gave up\n");
            CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));  // the next step starts clean
            CK(cudaStreamSynchronize(h->stream));
            return FVLBM_ERR_TIMEOUT;
        }
        stats->steps = h->steps;
        stats->residual = 0;
        stats->mass = 0;
        stats->diverged = 0;
        for (int q = 0; q < h->ninst; ++q) {
            const double num = sums[4 * q], den = sums[4 * q + 1];
            const double e = den > 0 ? std::sqrt(num) / std::sqrt(den) : std::sqrt(num);
            stats->residual = std::max(stats->residual, e);
            stats->mass += sums[4 * q + 2];
            if (sums[4 * q + 3] != 0.0 || !std::isfinite(e)) stats->diverged = 1;
        }
        if (stats->diverged) {
            if (h->rollback && h->rollback_step >= 0) {  // back to the last finite state
                size_t off = 0;
                for (auto &e : state_regions(h)) {
                    CK(cudaMemcpyAsync(e.first, static_cast<char *>(h->rollback) + off, e.second,
                                       cudaMemcpyDeviceToDevice, h->stream));
                    off += e.second;
                }
                CK(cudaStreamSynchronize(h->stream));
                h->steps = h->rollback_step;
                h->turb = h->rollback_turb;
                stats->steps = h->steps;
            }
            return FVLBM_ERR_DIVERGED;
        }
        if (h->rollback && (h->rollback_last < 0 || h->steps - h->rollback_last >= h->rollback_every)) {
            size_t off = 0;
            for (auto &e : state_regions(h)) {
                CK(cudaMemcpyAsync(static_cast<char *>(h->rollback) + off, e.first, e.second,
                                   cudaMemcpyDeviceToDevice, h->stream));
                off += e.second;
            }
            h->rollback_step = h->rollback_last = h->steps;
            h->rollback_turb = h->turb;
        }
    }
    return FVLBM_OK;
}

int fvlbm_get_f(fvlbm_handle *h, int instance, double *f) {
    if (!h || instance < -1 || instance >= h->ninst || !f) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    if (instance == -1) {
        const int n = h->total_nc;
        int rc = io_buffer(h, sizeof(double) * kQ * n);
        if (rc) return rc;
        const int nb = (n + 255) / 256;
        dispatch(h->precision, [&](auto z_) {
            using T = decltype(z_);
            k_gather_f_all<T><<<nb, 256, 0, h->stream>>>(static_cast<T *>(h->fn), h->d_all_map, n,
                                                              h->np, h->d_tile_inst, h->d_ip, h->d_io);
        });
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(f, h->d_io, sizeof(double) * kQ * n, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return FVLBM_OK;
    }
    const InstInfo &I = h->inst[instance];
    int rc = io_buffer(h, sizeof(double) * kQ * I.nc);
    if (rc) return rc;
    const int po = perm_offset(h, instance);
    const int nb = (I.nc + 255) / 256;
    dispatch(h->precision, [&](auto z_) {
        using T = decltype(z_);
        k_gather_f<T><<<nb, 256, 0, h->stream>>>(static_cast<T *>(h->fn), h->d_perm + po,
                                                      I.cell_off, I.nc, I.rho0, h->np, h->d_io);
    });
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(f, h->d_io, sizeof(double) * kQ * I.nc, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FVLBM_OK;
}

int fvlbm_set_f(fvlbm_handle *h, int instance, const double *f) {
    if (!h || instance < -1 || instance >= h->ninst || !f) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    const size_t n = io_cells(h, instance);
    int rc = io_buffer(h, sizeof(double) * kQ * n);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->d_io, f, sizeof(double) * kQ * n, cudaMemcpyHostToDevice, h->stream));
    scatter_state_dev(h, instance, static_cast<const double *>(h->d_io));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return FVLBM_OK;
}

int fvlbm_get_fields(fvlbm_handle *h, int instance, double *rho, double *u, double *v, double *k,
                     double *omega, double *nut) {
    if (!h || instance < -1 || instance >= h->ninst) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    const size_t n = io_cells(h, instance);
    int rc = io_buffer(h, sizeof(double) * 6 * n);
    if (rc) return rc;
    double *dst[6] = {rho, u, v, k, omega, nut};
    gather_fields_dev(h, instance, field_mask(dst), h->d_io);
    CK(cudaGetLastError());
    for (int q = 0; q < 6; ++q)
        if (dst[q])
            CK(cudaMemcpyAsync(dst[q], h->d_io + q * n, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FVLBM_OK;
}

// ---- cell lists of one instance (halo exchange of a partitioned mesh)
// Stages the list in the I/O buffer and maps it to internal ids: d_map receives them, d_vals
// the first byte after them (vals_bytes of room).  BAD_PARAM for an id outside the instance.
static int stage_cells(fvlbm_handle *h, int instance, int n, const int *cells, size_t vals_bytes,
                int **d_map, char **d_vals) {
    const InstInfo &I = h->inst[instance];
    for (int j = 0; j < n; ++j)
        if (cells[j] < 0 || cells[j] >= I.nc) return FVLBM_ERR_BAD_PARAM;
    const size_t ids = (2 * sizeof(int) * static_cast<size_t>(n) + 15) / 16 * 16;
    int rc = io_buffer(h, ids + vals_bytes);
    if (rc) return rc;
    int *d_cells = reinterpret_cast<int *>(h->d_io);
    *d_map = d_cells + n;
    *d_vals = reinterpret_cast<char *>(h->d_io) + ids;
    CK(cudaMemcpyAsync(d_cells, cells, sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
    k_cell_map<<<(n + 255) / 256, 256, 0, h->stream>>>(h->d_all_map + perm_offset(h, instance), d_cells, n,
                                                       *d_map);
    CK(cudaGetLastError());
    return FVLBM_OK;
}

int fvlbm_get_cells(fvlbm_handle *h, int instance, int n, const int *cells, double *f, double *k,
                    double *omega, double *nut) {
    if (!h || instance < 0 || instance >= h->ninst || n < 0 || (n > 0 && !cells)) return FVLBM_ERR_BAD_PARAM;
    if (n == 0) return FVLBM_OK;
    CK(cudaSetDevice(h->device));
    const bool turb = k || omega || nut;
    const size_t nf = static_cast<size_t>(n) * kQ, nt = 3 * static_cast<size_t>(n);
    int *d_map = nullptr;
    char *d_vals = nullptr;
    int rc = stage_cells(h, instance, n, cells, sizeof(double) * (nf + nt), &d_map, &d_vals);
    if (rc) return rc;
    double *d_f = reinterpret_cast<double *>(d_vals), *d_t = d_f + nf;
    const InstInfo &I = h->inst[instance];
    dispatch(h->precision, [&](auto z_) {
        using T = decltype(z_);
        const int c = h->turb;
        k_get_cells<T><<<(n + 255) / 256, 256, 0, h->stream>>>(
            static_cast<const T *>(h->fn), turb ? static_cast<const T *>(h->kk[c]) : nullptr,
            static_cast<const T *>(h->ww[c]), static_cast<const T *>(h->nut[c]), d_map, n, I.rho0, h->np,
            d_f, d_t);
    });
    CK(cudaGetLastError());
    std::vector<double> t(turb ? nt : 0);
    if (f) CK(cudaMemcpyAsync(f, d_f, sizeof(double) * nf, cudaMemcpyDeviceToHost, h->stream));
    if (turb) CK(cudaMemcpyAsync(t.data(), d_t, sizeof(double) * nt, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int j = 0; turb && j < n; ++j) {
        if (k) k[j] = t[j];
        if (omega) omega[j] = t[n + j];
        if (nut) nut[j] = t[2 * static_cast<size_t>(n) + j];
    }
    return FVLBM_OK;
}

int fvlbm_set_cells(fvlbm_handle *h, int instance, int n, const int *cells, const double *f,
                    const double *k, const double *omega, const double *nut) {
    if (!h || instance < 0 || instance >= h->ninst || n < 0 || (n > 0 && !cells)) return FVLBM_ERR_BAD_PARAM;
    const bool turb = k || omega || nut;
    if (turb && !(k && omega && nut)) return FVLBM_ERR_BAD_PARAM;
    if (n == 0) return FVLBM_OK;
    CK(cudaSetDevice(h->device));
    const size_t nf = static_cast<size_t>(n) * kQ, nt = 3 * static_cast<size_t>(n);
    int *d_map = nullptr;
    char *d_vals = nullptr;
    int rc = stage_cells(h, instance, n, cells, sizeof(double) * (nf + nt), &d_map, &d_vals);
    if (rc) return rc;
    double *d_f = reinterpret_cast<double *>(d_vals), *d_t = d_f + nf;
    if (f) CK(cudaMemcpyAsync(d_f, f, sizeof(double) * nf, cudaMemcpyHostToDevice, h->stream));
    if (turb) {
        std::vector<double> t(nt);
        std::copy(k, k + n, t.begin());
        std::copy(omega, omega + n, t.begin() + n);
        std::copy(nut, nut + n, t.begin() + 2 * static_cast<size_t>(n));
        CK(cudaMemcpyAsync(d_t, t.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));  // t is a local buffer
    }
    dispatch(h->precision, [&](auto z_) {
        using T = decltype(z_);
        const int c = h->turb;
        if (f)  // f^n, the macros and f^(1) of the coming step, as fvlbm_set_f
            k_scatter_list<T, double><<<(n + 255) / 256, 256, 0, h->stream>>>(
                static_cast<T *>(h->fn), static_cast<T *>(h->mac), static_cast<T *>(frel_target(h)),
                static_cast<const T *>(h->tau), d_map, n, geo_of<T>(h), d_f);
        if (turb)
            k_set_turb<T><<<(n + 255) / 256, 256, 0, h->stream>>>(static_cast<T *>(h->kk[c]),
                                                                 static_cast<T *>(h->ww[c]),
                                                                 static_cast<T *>(h->nut[c]), d_map, n, d_t);
    });
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return FVLBM_OK;
}

int fvlbm_set_wall_distance(fvlbm_handle *h, int instance, const double *d) {
    if (!h || instance < 0 || instance >= h->ninst || !d) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    const InstInfo &I = h->inst[instance];
    for (int j = 0; j < I.nc; ++j)
        if (!(d[j] > 0.0)) return FVLBM_ERR_BAD_PARAM;
    int rc = io_buffer(h, sizeof(double) * std::max(I.nc, 1));
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->d_io, d, sizeof(double) * I.nc, cudaMemcpyHostToDevice, h->stream));
    dispatch(h->precision, [&](auto z_) {
        using T = decltype(z_);
        k_set_wdist<T><<<(I.nc + 255) / 256, 256, 0, h->stream>>>(static_cast<T *>(h->wdist),
                                                                  h->d_all_map + perm_offset(h, instance),
                                                                  I.nc, h->d_io);
    });
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return FVLBM_OK;
}

int fvlbm_set_exchange_list(fvlbm_handle *h, int instance, int n, const int *cells, int *list_id) {
    if (!h || instance < 0 || instance >= h->ninst || n < 0 || (n > 0 && !cells) || !list_id)
        return FVLBM_ERR_BAD_PARAM;
    const InstInfo &I = h->inst[instance];
    for (int j = 0; j < n; ++j)
        if (cells[j] < 0 || cells[j] >= I.nc) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    fvlbm_handle::XList L{instance, n, nullptr};
    int rc = dalloc(h, reinterpret_cast<void **>(&L.d_map), sizeof(int) * 2 * std::max(n, 1));
    if (rc) return rc;
    if (n > 0) {
        int *d_cells = L.d_map + n;
        CK(cudaMemcpyAsync(d_cells, cells, sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
        k_cell_map<<<(n + 255) / 256, 256, 0, h->stream>>>(h->d_all_map + perm_offset(h, instance), d_cells, n,
                                                           L.d_map);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->stream));
    }
    *list_id = static_cast<int>(h->xlists.size());
    h->xlists.push_back(L);
    return FVLBM_OK;
}

int fvlbm_pack_cells_dev(fvlbm_handle *h, int list_id, double *vals) {
    if (!h || list_id < 0 || list_id >= static_cast<int>(h->xlists.size())) return FVLBM_ERR_BAD_PARAM;
    const auto &L = h->xlists[list_id];
    if (L.n == 0) return FVLBM_OK;
    if (!vals) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    dispatch(h->precision, [&](auto z_) {
        using T = decltype(z_);
        const int c = h->turb;
        k_pack_cells<T><<<(L.n + 255) / 256, 256, 0, h->stream>>>(
            static_cast<const T *>(h->fn), static_cast<const T *>(h->kk[c]), static_cast<const T *>(h->ww[c]),
            static_cast<const T *>(h->nut[c]), L.d_map, L.n, geo_of<T>(h), vals);
    });
    CK(cudaGetLastError());
    return FVLBM_OK;
}

int fvlbm_unpack_cells_dev(fvlbm_handle *h, int list_id, const double *vals) {
    if (!h || list_id < 0 || list_id >= static_cast<int>(h->xlists.size())) return FVLBM_ERR_BAD_PARAM;
    const auto &L = h->xlists[list_id];
    if (L.n == 0) return FVLBM_OK;
    if (!vals) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    dispatch(h->precision, [&](auto z_) {
        using T = decltype(z_);
        const int c = h->turb;
        k_unpack_cells<T><<<(L.n + 255) / 256, 256, 0, h->stream>>>(
            static_cast<T *>(h->fn), static_cast<T *>(h->mac), static_cast<T *>(frel_target(h)),
            static_cast<const T *>(h->tau), static_cast<T *>(h->kk[c]), static_cast<T *>(h->ww[c]),
            static_cast<T *>(h->nut[c]), L.d_map, L.n, geo_of<T>(h), vals);
    });
    CK(cudaGetLastError());
    return FVLBM_OK;
}

int fvlbm_forces_edges(fvlbm_handle *h, int instance, double *fxy) {
    if (!fxy) return FVLBM_ERR_BAD_PARAM;
    double out[4];
    return forces_impl(h, instance, 0.0, out, nullptr, nullptr, nullptr, fxy);
}

int fvlbm_set_f_async(fvlbm_handle *h, int instance, const double *f) {
    if (!h || instance < -1 || instance >= h->ninst || !f) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    int rc = async_init(h);
    if (rc) return rc;
    auto &A = h->aio;
    const int slot = A.in_next;
    A.in_next ^= 1;
    const size_t bytes = sizeof(double) * kQ * io_cells(h, instance);
    if ((rc = async_slot(h, &A.d_in[slot], &A.in_cap[slot], bytes))) return rc;
    CK(cudaStreamWaitEvent(A.s_in, A.in_free[slot], 0));  // the slot's last scatter has run
    CK(cudaMemcpyAsync(A.d_in[slot], f, bytes, cudaMemcpyHostToDevice, A.s_in));
    CK(cudaEventRecord(A.in_ready[slot], A.s_in));
    CK(cudaStreamWaitEvent(h->stream, A.in_ready[slot], 0));
    scatter_state_dev(h, instance, static_cast<const double *>(A.d_in[slot]));
    CK(cudaGetLastError());
    CK(cudaEventRecord(A.in_free[slot], h->stream));
    return FVLBM_OK;
}

int fvlbm_get_fields_async(fvlbm_handle *h, int instance, double *rho, double *u, double *v, double *k,
                           double *omega, double *nut) {
    if (!h || instance < -1 || instance >= h->ninst) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    int rc = async_init(h);
    if (rc) return rc;
    auto &A = h->aio;
    const int slot = A.out_next;
    A.out_next ^= 1;
    const size_t n = io_cells(h, instance);
    if ((rc = async_slot(h, &A.d_out[slot], &A.out_cap[slot], sizeof(double) * 6 * n))) return rc;
    CK(cudaStreamWaitEvent(h->stream, A.out_free[slot], 0));  // the slot's last copy-out is done
    double *dst[6] = {rho, u, v, k, omega, nut};
    gather_fields_dev(h, instance, field_mask(dst), A.d_out[slot]);
    CK(cudaGetLastError());
    CK(cudaEventRecord(A.out_ready[slot], h->stream));
    CK(cudaStreamWaitEvent(A.s_out, A.out_ready[slot], 0));
    for (int q = 0; q < 6; ++q)
        if (dst[q])
            CK(cudaMemcpyAsync(dst[q], A.d_out[slot] + q * n, sizeof(double) * n, cudaMemcpyDeviceToHost,
                               A.s_out));
    CK(cudaEventRecord(A.out_free[slot], A.s_out));
    return FVLBM_OK;
}

int fvlbm_get_fdev_f32(fvlbm_handle *h, int instance, float *fdev) {
    if (!h || instance < -1 || instance >= h->ninst || !fdev) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    const int n = static_cast<int>(io_cells(h, instance));
    const int po = instance == -1 ? 0 : perm_offset(h, instance);
    int rc = io_buffer(h, sizeof(float) * kQ * static_cast<size_t>(n));
    if (rc) return rc;
    float *buf = reinterpret_cast<float *>(h->d_io);
    dispatch(h->precision, [&](auto z_) {
        using T = decltype(z_);
        k_gather_fdev32<T><<<(n + 255) / 256, 256, 0, h->stream>>>(static_cast<const T *>(h->fn),
                                                                   h->d_all_map + po, n, h->np, buf);
    });
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(fdev, buf, sizeof(float) * kQ * static_cast<size_t>(n), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FVLBM_OK;
}

int fvlbm_set_fdev_f32_async(fvlbm_handle *h, int instance, const float *fdev) {
    if (!h || instance < -1 || instance >= h->ninst || !fdev) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    int rc = async_init(h);
    if (rc) return rc;
    auto &A = h->aio;
    const int slot = A.in_next;
    A.in_next ^= 1;
    const size_t bytes = sizeof(float) * kQ * io_cells(h, instance);
    if ((rc = async_slot(h, &A.d_in[slot], &A.in_cap[slot], bytes))) return rc;
    float *buf = reinterpret_cast<float *>(A.d_in[slot]);
    CK(cudaStreamWaitEvent(A.s_in, A.in_free[slot], 0));
    CK(cudaMemcpyAsync(buf, fdev, bytes, cudaMemcpyHostToDevice, A.s_in));
    CK(cudaEventRecord(A.in_ready[slot], A.s_in));
    CK(cudaStreamWaitEvent(h->stream, A.in_ready[slot], 0));
    scatter_state_dev(h, instance, static_cast<const float *>(buf));
    CK(cudaGetLastError());
    CK(cudaEventRecord(A.in_free[slot], h->stream));
    return FVLBM_OK;
}

int fvlbm_wait(fvlbm_handle *h) {
    if (!h) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    if (h->aio.init) {
        CK(cudaStreamSynchronize(h->aio.s_in));
        CK(cudaStreamSynchronize(h->aio.s_out));
    }
    return FVLBM_OK;
}

int fvlbm_forces(fvlbm_handle *h, int instance, double *out, double *cp) {
    return forces_impl(h, instance, 0.0, out, nullptr, cp);
}

int fvlbm_adjoint(fvlbm_handle *h, int instance, int n_steps, const double *w, double *J, double *dJ_df,
                  double *dJ_dbedge_val, double *dJ_dxy) {
    return adjoint_impl(h, instance, n_steps, w, J, dJ_df, dJ_dbedge_val, dJ_dxy);
}

// Parameter gradient of J = w[0] C_D + w[1] C_L (see the header): one adjoint solve, then
// the chain rule through the parameter map on the host.
//   alpha: far-field velocity (u_b, v_b) rotated by alpha, d(u_b, v_b)/d alpha = (-v_b, u_b),
//          and the drag / lift axes, dC_D/d alpha = C_L, dC_L/d alpha = -C_D;
//   ratio: omega_b = k_b / (nu ratio) on far-field and inlet edges with k_b > 0,
//          d omega_b / d ratio = -omega_b / ratio = -omega_b^2 nu / k_b;
//   wall node j displaced along n_j: dJ/d s_j = dJ/d(x, y)_node . n_j.
int fvlbm_adjoint_params(fvlbm_handle *h, int instance, int n_steps, const double *w, int n_wall,
                         const int *wall_nodes, const double *wall_normals, double *J, double *cdcl,
                         double *dJ_dalpha, double *dJ_dratio, double *dJ_dwall) {
    if (!h || instance < 0 || instance >= h->ninst || !w || n_wall < 0 ||
        (n_wall > 0 && (!wall_nodes || !wall_normals || !dJ_dwall)))
        return FVLBM_ERR_BAD_PARAM;
    if (h->precision != FVLBM_FP64) return FVLBM_ERR_NOT_SUPPORTED;
    const InstInfo &I = h->inst[instance];
    if (!I.mesh) return FVLBM_ERR_NOT_SUPPORTED;
    const MeshCopy &mc = *I.mesh;
    for (int j = 0; j < n_wall; ++j)
        if (wall_nodes[j] < 0 || wall_nodes[j] >= I.n_nodes) return FVLBM_ERR_BAD_PARAM;
    const int nbe = I.n_bedges_in;
    std::vector<double> dbv(5 * static_cast<size_t>(std::max(nbe, 1)), 0.0);
    std::vector<double> dxy;
    if (n_wall > 0) dxy.assign(2 * static_cast<size_t>(I.n_nodes), 0.0);
    double Jv = 0.0, cc[2] = {0.0, 0.0};
    const int rc = adjoint_impl(h, instance, n_steps, w, &Jv, nullptr, dbv.data(),
                                n_wall > 0 ? dxy.data() : nullptr, cc);
    if (rc) return rc;
    double da = w[0] * cc[1] - w[1] * cc[0], dr = 0.0;
    for (int b = 0; b < nbe; ++b) {
        const int t = mc.btype[b];
        const double *v = &mc.bval[5 * static_cast<size_t>(b)];
        const double *g = &dbv[5 * static_cast<size_t>(b)];
        if (t == FVLBM_BC_FARFIELD) da += g[1] * (-v[2]) + g[2] * v[1];
        if ((t == FVLBM_BC_FARFIELD || t == FVLBM_BC_INLET) && v[3] > 0.0)
            dr += g[4] * (-v[4] * v[4] * I.nu / v[3]);
    }
    for (int j = 0; j < n_wall; ++j) {
        const size_t nd = static_cast<size_t>(wall_nodes[j]);
        dJ_dwall[j] = dxy[2 * nd] * wall_normals[2 * j] + dxy[2 * nd + 1] * wall_normals[2 * j + 1];
    }
    if (J) *J = Jv;
    if (cdcl) {
        cdcl[0] = cc[0];
        cdcl[1] = cc[1];
    }
    if (dJ_dalpha) *dJ_dalpha = da;
    if (dJ_dratio) *dJ_dratio = dr;
    return FVLBM_OK;
}

int fvlbm_fv_items(fvlbm_handle *h, int *nitem, int *n_split, int *n_overflow) {
    if (!h || !nitem || !n_split || !n_overflow) return FVLBM_ERR_BAD_PARAM;
    *nitem = h->fv.ok ? h->fv.nitem : 0;
    *n_split = h->fv.ok ? h->fv.n_split : 0;
    *n_overflow = h->fv.ok ? h->fv.n_ovf : 0;
    return FVLBM_OK;
}

int fvlbm_set_wait_limit(fvlbm_handle *h, long long polls) {
    if (!h || polls < 0) return FVLBM_ERR_BAD_PARAM;
    h->wait_first = polls;
    for (int k = 0; k < 3; ++k)  // captured graphs bake the kernel arguments
        if (h->graph[k]) {
            cudaGraphExecDestroy(h->graph[k]);
            h->graph[k] = nullptr;
        }
    return FVLBM_OK;
}

int fvlbm_set_adjoint_budget(fvlbm_handle *h, long long bytes) {
    if (!h || bytes < 0) return FVLBM_ERR_BAD_PARAM;
    h->adj_budget = static_cast<size_t>(bytes);
    return FVLBM_OK;
}

int fvlbm_tangent_seed(fvlbm_handle *h, int instance, const double *dbedge_val, const double *df) {
    if (!h || instance < 0 || instance >= h->ninst) return FVLBM_ERR_BAD_PARAM;
    if (h->precision != FVLBM_FP64_TANGENT) return FVLBM_ERR_NOT_SUPPORTED;
    CK(cudaSetDevice(h->device));
    const InstInfo &I = h->inst[instance];
    if (dbedge_val && I.nb > 0) {
        // boundary values are field-major [5][nbt]; the instance's faces are one run per field
        std::vector<Dual> bv(static_cast<size_t>(5) * I.nb);
        Dual *dev = static_cast<Dual *>(h->bval);
        for (int c = 0; c < 5; ++c)
            CK(cudaMemcpyAsync(bv.data() + static_cast<size_t>(c) * I.nb,
                               dev + static_cast<size_t>(c) * h->nbt + I.bface_off, sizeof(Dual) * I.nb,
                               cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int b = 0; b < I.nb; ++b)
            for (int c = 0; c < 5; ++c)
                bv[static_cast<size_t>(c) * I.nb + b].d = dbedge_val[5 * static_cast<size_t>(I.bedge_of[b]) + c];
        for (int c = 0; c < 5; ++c)
            CK(cudaMemcpyAsync(dev + static_cast<size_t>(c) * h->nbt + I.bface_off,
                               bv.data() + static_cast<size_t>(c) * I.nb, sizeof(Dual) * I.nb,
                               cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    if (df && I.nc > 0) {
        const size_t bytes = sizeof(double) * kQ * static_cast<size_t>(I.nc);
        int rc = io_buffer(h, bytes);
        if (rc) return rc;
        CK(cudaMemcpyAsync(h->d_io, df, bytes, cudaMemcpyHostToDevice, h->stream));
        const int nb = (I.nc + 255) / 256;
        k_seed_df<<<nb, 256, 0, h->stream>>>(static_cast<Dual *>(h->fn), static_cast<Dual *>(h->mac),
                                             h->d_perm + perm_offset(h, instance), I.cell_off, I.nc, I.rho0,
                                             h->np, h->d_io);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->stream));
    }
    return FVLBM_OK;
}

int fvlbm_tangent_seed_nodes(fvlbm_handle *h, int instance, const double *dxy) {
    if (!h || instance < 0 || instance >= h->ninst || !dxy) return FVLBM_ERR_BAD_PARAM;
    if (h->precision != FVLBM_FP64_TANGENT) return FVLBM_ERR_NOT_SUPPORTED;
    CK(cudaSetDevice(h->device));
    const InstInfo &I = h->inst[instance];
    const MeshCopy &mc = *I.mesh;
    // the instance's preprocessing again, on node positions that carry d(x, y)/dp
    std::vector<Dual> xyd(mc.xy.size());
    for (size_t k = 0; k < xyd.size(); ++k) xyd[k] = Dual(mc.xy[k], dxy[k]);
    const fvlbm_mesh M{I.n_nodes, mc.xy.data(), I.nc, mc.cell_ptr.data(), mc.cell_nodes.data()};
    const int nbe = static_cast<int>(mc.btype.size());
    const fvlbm_bc B{nbe, mc.bnodes.data(), mc.btype.data(), mc.bval.data(),
                     static_cast<int>(mc.ppairs.size() / 2), mc.ppairs.data(), mc.pshift.data()};
    PreparedT<Dual> D;
    std::string why;
    const int rc = prepare_instance_t<Dual>(M, B, mc.params, xyd.data(), &D, &why);
    if (rc) {
        fprintf(stderr, "fvlbm_tangent_seed_nodes: %s\n", why.c_str());
        return rc;
    }
    if (D.perm != mc.perm || D.np != I.np || D.nb != I.nb) return FVLBM_ERR_NOT_SUPPORTED;
    // Derivative parts into the device arrays.  dst holds ncomp runs of n values at
    // dst[c * stride + off]; get(c, k) is the Dual of component c, item k.
    const size_t np = h->np, nbt = h->nbt;
    auto put = [&](void *dst, int ncomp, size_t stride, size_t off, size_t n, auto get) -> int {
        if (n == 0) return FVLBM_OK;
        std::vector<Dual> run(n);
        Dual *dev = static_cast<Dual *>(dst);
        for (int c = 0; c < ncomp; ++c) {
            CK(cudaMemcpy(run.data(), dev + c * stride + off, n * sizeof(Dual), cudaMemcpyDeviceToHost));
            for (size_t k = 0; k < n; ++k) run[k].d = get(c, k).d;
            CK(cudaMemcpy(dev + c * stride + off, run.data(), n * sizeof(Dual), cudaMemcpyHostToDevice));
        }
        return FVLBM_OK;
    };
    CK(cudaStreamSynchronize(h->stream));
    const size_t pn = I.np, co = I.cell_off, nb = I.nb, bo = I.bface_off;
    int e = 0;
    e = e ? e : put(h->sn, 8, np, co, pn, [&](int c, size_t k) { return D.sn[c * pn + k]; });
    e = e ? e : put(h->lsq, 8, np, co, pn, [&](int c, size_t k) { return D.lsq[c * pn + k]; });
    e = e ? e : put(h->rown, 8, np, co, pn, [&](int c, size_t k) { return D.rown[c * pn + k]; });
    e = e ? e : put(h->rnbr, 8, np, co, pn, [&](int c, size_t k) { return D.rnbr[c * pn + k]; });
    e = e ? e : put(h->dinv, 4, np, co, pn, [&](int c, size_t k) { return D.dinv[c * pn + k]; });
    e = e ? e : put(h->area, 1, np, co, pn, [&](int, size_t k) { return D.area[k]; });
    e = e ? e : put(h->wdist, 1, np, co, pn, [&](int, size_t k) { return D.wdist[k]; });
    e = e ? e : put(h->bnrm, 2, nbt, bo, nb, [&](int c, size_t f) { return D.bnrm[2 * f + c]; });
    e = e ? e : put(h->blen, 1, nbt, bo, nb, [&](int, size_t f) { return D.blen[f]; });
    return e;
}

int fvlbm_get_f_tangent(fvlbm_handle *h, int instance, double *df) {
    if (!h || instance < 0 || instance >= h->ninst || !df) return FVLBM_ERR_BAD_PARAM;
    if (h->precision != FVLBM_FP64_TANGENT) return FVLBM_ERR_NOT_SUPPORTED;
    CK(cudaSetDevice(h->device));
    const InstInfo &I = h->inst[instance];
    if (I.nc == 0) return FVLBM_OK;
    const size_t bytes = sizeof(double) * kQ * static_cast<size_t>(I.nc);
    int rc = io_buffer(h, bytes);
    if (rc) return rc;
    const int nb = (I.nc + 255) / 256;
    k_gather_df<<<nb, 256, 0, h->stream>>>(static_cast<const Dual *>(h->fn), h->d_perm + perm_offset(h, instance),
                                           I.cell_off, I.nc, h->np, h->d_io);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(df, h->d_io, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FVLBM_OK;
}

int fvlbm_forces_tangent(fvlbm_handle *h, int instance, double dalpha, double *out, double *dout) {
    if (!h || !dout) return FVLBM_ERR_BAD_PARAM;
    if (h->precision != FVLBM_FP64_TANGENT) return FVLBM_ERR_NOT_SUPPORTED;
    return forces_impl(h, instance, dalpha, out, dout, nullptr);
}

int fvlbm_info(fvlbm_handle *h, int instance, int *n_cells, int *n_bedges, double *dt) {
    if (!h || instance < -1 || instance >= h->ninst) return FVLBM_ERR_BAD_PARAM;
    if (instance == -1) {  // totals over all instances
        int nbe = 0;
        for (const auto &I : h->inst) nbe += I.n_bedges_in;
        if (n_cells) *n_cells = h->total_nc;
        if (n_bedges) *n_bedges = nbe;
        if (dt) *dt = 0.0;
        return FVLBM_OK;
    }
    const InstInfo &I = h->inst[instance];
    if (n_cells) *n_cells = I.nc;
    if (n_bedges) *n_bedges = I.n_bedges_in;
    if (dt) *dt = I.dt;
    return FVLBM_OK;
}

int fvlbm_footprint(fvlbm_handle *h, long long *device_bytes, int *lps) {
    if (!h) return FVLBM_ERR_BAD_PARAM;
    if (device_bytes) *device_bytes = static_cast<long long>(h->device_bytes);
    if (lps) *lps = launches_per_step(h);
    return FVLBM_OK;
}

int fvlbm_profile_kernels(fvlbm_handle *h, int n_steps, int max_kernels, char *names, double *ms,
                          int *launches) {
    if (!h || n_steps <= 0) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    h->profiling = true;
    h->timers.clear();
    for (int k = 0; k < n_steps; ++k) enqueue(h, false);
    h->steps += n_steps;
    h->profiling = false;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    for (auto &pe : h->pending) {
        float t = 0;
        if (e == cudaSuccess) cudaEventElapsedTime(&t, pe.second.first, pe.second.second);
        h->timers[pe.first].ms += t;
        h->timers[pe.first].launches += 1;
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    h->pending.clear();
    if (e != cudaSuccess) return cuda_fail(e);
    int nk = 0;
    for (const auto &t : h->timers) {
        if (t.launches == 0) continue;
        if (nk < max_kernels) {
            if (names) {
                std::memset(names + 32 * nk, 0, 32);
                std::strncpy(names + 32 * nk, t.name.c_str(), 31);
            }
            if (ms) ms[nk] = t.ms;
            if (launches) launches[nk] = t.launches;
        }
        ++nk;
    }
    return std::min(nk, max_kernels);
}

int fvlbm_autotune(fvlbm_handle *h, int trial_steps, int *chosen, double *ms_per_step) {
    if (!h || trial_steps <= 0) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    if (ms_per_step)
        for (int c = 0; c < 4; ++c) ms_per_step[c] = -1.0;
    if (h->scheme != 0 || (!h->hs[0].ok && !h->hs[1].ok && !h->fv.ok)) {  // nothing to choose
        if (chosen) *chosen = h->config;
        return FVLBM_OK;
    }
    // snapshot of the state a step reads (the rest is scratch)
    const std::vector<std::pair<void *, size_t>> st = state_regions(h);
    size_t total = 0;
    for (auto &e : st) total += e.second;
    char *snap = nullptr;
    CK(cudaMalloc(reinterpret_cast<void **>(&snap), total));
    auto copy_all = [&](bool save) {
        size_t off = 0;
        for (auto &e : st) {
            if (save)
                cudaMemcpyAsync(snap + off, e.first, e.second, cudaMemcpyDeviceToDevice, h->stream);
            else
                cudaMemcpyAsync(e.first, snap + off, e.second, cudaMemcpyDeviceToDevice, h->stream);
            off += e.second;
        }
    };
    copy_all(true);
    const int turb0 = h->turb;
    const long long steps0 = h->steps;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    int best_c = h->config;
    cudaError_t err = cudaSuccess;
    for (int c = 0; c < 4 && err == cudaSuccess; ++c) {
        if (c < 2 && (!h->hs[c].ok || h->precision == FVLBM_FP32_DEV)) continue;  // see create
        if (c == 3 && !h->fv.ok) continue;
        h->config = c;
        for (int k = 0; k < 2; ++k) enqueue(h, false);  // warm-up
        cudaEventRecord(e0, h->stream);
        for (int k = 0; k < trial_steps; ++k) enqueue(h, false);
        cudaEventRecord(e1, h->stream);
        err = cudaStreamSynchronize(h->stream);
        float ms = 0.f;
        if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        const double per = double(ms) / trial_steps;
        if (ms_per_step) ms_per_step[c] = per;
        if (per < best) {
            best = per;
            best_c = c;
        }
        copy_all(false);
        h->turb = turb0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
    cudaFree(snap);
    h->config = best_c;
    h->steps = steps0;
    // The two-pass kernels do not keep f^(1) of the coming step: if they ran before this call,
    // the restored snapshot holds a stale one.  Relax it again from f^n for the fused stages
    // (bitwise what stage 3 writes for laminar instances; SST instances redo it every step).
    if (best_c != 2 && err == cudaSuccess)
        dispatch(h->precision, [&](auto z_) { relax_all<decltype(z_)>(h); });
    for (int k = 0; k < 3; ++k)  // captured graphs bake the old configuration
        if (h->graph[k]) {
            cudaGraphExecDestroy(h->graph[k]);
            h->graph[k] = nullptr;
        }
    if (chosen) *chosen = best_c;
    if (err != cudaSuccess) return cuda_fail(err);
    CK(cudaGetLastError());
    return FVLBM_OK;
}

int fvlbm_state_bytes(fvlbm_handle *h, long long *bytes) {
    if (!h || !bytes) return FVLBM_ERR_BAD_PARAM;
    *bytes = static_cast<long long>(sizeof(StateHeader) + state_bytes(h));
    return FVLBM_OK;
}

int fvlbm_save_state(fvlbm_handle *h, void *buf, long long bytes) {
    if (!h || !buf || bytes < static_cast<long long>(sizeof(StateHeader) + state_bytes(h)))
        return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    StateHeader hd{};
    std::memcpy(hd.magic, "FVLBMST", 8);
    hd.version = 1;
    hd.precision = h->precision;
    hd.np = h->np;
    hd.ninst = h->ninst;
    hd.turb = h->turb;
    hd.steps = h->steps;
    hd.order_hash = h->order_hash;
    hd.payload = state_bytes(h);
    std::memcpy(buf, &hd, sizeof(hd));
    char *dst = static_cast<char *>(buf) + sizeof(hd);
    for (auto &e : state_regions(h)) {
        CK(cudaMemcpyAsync(dst, e.first, e.second, cudaMemcpyDeviceToHost, h->stream));
        dst += e.second;
    }
    CK(cudaStreamSynchronize(h->stream));
    return FVLBM_OK;
}

int fvlbm_load_state(fvlbm_handle *h, const void *buf, long long bytes) {
    if (!h || !buf || bytes < static_cast<long long>(sizeof(StateHeader))) return FVLBM_ERR_BAD_PARAM;
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, "FVLBMST", 8) != 0 || hd.version != 1 || hd.precision != h->precision ||
        hd.np != h->np || hd.ninst != h->ninst || hd.order_hash != h->order_hash ||
        hd.payload != state_bytes(h) || bytes < static_cast<long long>(sizeof(hd) + hd.payload)) {
        fprintf(stderr, "fvlbm_load_state: the blob does not match this handle\n");
        return FVLBM_ERR_BAD_PARAM;
    }
    CK(cudaSetDevice(h->device));
    const char *src = static_cast<const char *>(buf) + sizeof(hd);
    for (auto &e : state_regions(h)) {
        CK(cudaMemcpyAsync(e.first, src, e.second, cudaMemcpyHostToDevice, h->stream));
        src += e.second;
    }
    // a blob saved under the face-value configuration holds no f^(1) of the coming step: the
    // other fused configurations relax it from f^n again (bitwise what they would have stored)
    if (h->config == 0 || h->config == 1)
        dispatch(h->precision, [&](auto z_) {
            if constexpr (kHasFused<decltype(z_)>) relax_all<decltype(z_)>(h);
        });
    CK(cudaStreamSynchronize(h->stream));
    h->steps = hd.steps;
    h->turb = hd.turb;
    return FVLBM_OK;
}

int fvlbm_set_rollback(fvlbm_handle *h, int every) {
    if (!h || every < 0) return FVLBM_ERR_BAD_PARAM;
    CK(cudaSetDevice(h->device));
    if (every == 0) {
        if (h->rollback) {
            cudaStreamSynchronize(h->stream);
            cudaFree(h->rollback);
            h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), h->rollback));
            h->device_bytes -= state_bytes(h);
            h->rollback = nullptr;
        }
    } else if (!h->rollback) {
        int rc = dalloc(h, &h->rollback, state_bytes(h));
        if (rc) return rc;
    }
    h->rollback_every = every;
    h->rollback_step = h->rollback_last = -1;
    return FVLBM_OK;
}

void fvlbm_destroy(fvlbm_handle *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

const char *fvlbm_strerror(int code) {
    switch (code) {
    case FVLBM_OK: return "ok";
    case FVLBM_ERR_BAD_MESH: return "bad mesh";
    case FVLBM_ERR_BAD_BC: return "bad boundary conditions";
    case FVLBM_ERR_BAD_PARAM: return "bad parameter";
    case FVLBM_ERR_OOM: return "out of device memory";
    case FVLBM_ERR_CUDA: return "CUDA runtime error";
    case FVLBM_ERR_DIVERGED: return "state diverged (NaN or Inf)";
    case FVLBM_ERR_NOT_SUPPORTED: return "not supported";
    case FVLBM_ERR_TIMEOUT: return "a bounded wait inside a kernel gave up";
    default: return "unknown error";
    }
}

}  // extern "C"
