// fvlbm_adjoint.cuh -- discrete adjoint (reverse mode) of the laminar FP64 time step, included
// into fvlbm_kernels.cu after the handle and its helpers.
//
// The map differentiated is the two-pass IMEX step exactly as the library runs it (Sec. 3.2,
// Steps 2-7 without Step 1): f^(1) = R(f^n) (Eq. (fnewstage), J = 1), three gradient + flux
// evaluations (Step 2, Eq. (advection)) and the stage algebra of the two accumulators.  Per step
//   s1 = R(f0);  a1 = A(s1);  (f2, B, C) = S1(f0, a1);  a2 = A(f2);  f3 = S2(B - dt/2 a2);
//   C' = C + dt/6 a2;  a3 = A(f3);  f^{n+1} = f3 + C' - dt/3 a3,
// with A(f) = sum over faces of (e . n dl / A) times the upwind linear face value built from
// the least-squares gradient, boundary faces taking the boundary values of Part I.  The adjoint
// runs these in reverse: the linear flux and gradient operators are transposed by gathering
// over each cell's faces (the neighbour's view of a shared face comes from its back slot), and
// the per-cell nonlinear maps (R, S1, S2, the boundary values) are transposed through their
// local Jacobians, evaluated column by column with the dual-number type of the tangent path.
// States are recomputed from checkpoints (every K-th state kept, K ~ sqrt(n_steps); one
// segment of K states rebuilt at a time), so the storage is about 2 sqrt(n_steps) states.

namespace fvlbm {

// ---- per-cell maps, written out exactly as the forward kernels evaluate them
template <class T>
__device__ __forceinline__ void adj_relax(const T *f0, T rho0, T dt, T tau, T *s1) {
#pragma unroll
    for (int a = 0; a < kQ; ++a) s1[a] = f0[a];
    relax9(s1, rho0, dt, tau);
}

// Stage-1 algebra of the two-pass path (stage_algebra, J = 1, f^n given).
template <class T>
__device__ __forceinline__ void adj_stage1(const T *f0, const T *acc, T rho0, T dt, T tau, T *f2, T *B,
                                           T *C) {
    const T itau = T(1) / tau;
    const T dt6 = dt * T(1.0 / 6.0);
    T eq[kQ], X[kQ], dgc1[kQ], dr, r, u, v;
    const T z = dt * itau;
    const T zq = z * T(0.25);
    const T inv = T(1) / (T(1) + zq);
    moments(f0, rho0, dr, r, u, v);
    feq_dev(dr, r, u, v, eq);
    const T s1 = z * inv;
#pragma unroll
    for (int a = 0; a < kQ; ++a) dgc1[a] = (eq[a] - f0[a]) * s1;
#pragma unroll
    for (int a = 0; a < kQ; ++a) X[a] = f0[a] - T(0.5) * dt * acc[a];
    moments(X, rho0, dr, r, u, v);
    feq_dev(dr, r, u, v, eq);
    const T s2 = z * inv;
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        f2[a] = (X[a] + zq * eq[a]) * inv;
        const T dgc2 = (eq[a] - X[a]) * s2;
        B[a] = X[a] + T(1.0 / 3.0) * (dgc1[a] + dgc2);
        C[a] = dt6 * acc[a];
    }
}

// Stage-2 solve from X = B - dt/2 acc (stage_algebra, J = 2).
template <class T>
__device__ __forceinline__ void adj_stage2(const T *X, T rho0, T dt, T tau, T *f3) {
    const T itau = T(1) / tau;
    const T dt3 = dt * T(1.0 / 3.0);
    T eq[kQ], dr, r, u, v;
    moments(X, rho0, dr, r, u, v);
    feq_dev(dr, r, u, v, eq);
    const T zt = dt3 * itau;
    const T inv = T(1) / (T(1) + zt);
#pragma unroll
    for (int a = 0; a < kQ; ++a) f3[a] = (X[a] + zt * eq[a]) * inv;
}

// Boundary values of one face as a function of the owner's f and of (rho_b, u_b, v_b).
template <class T>
__device__ __forceinline__ void adj_bvals(int type, const T *bv3, T snx, T sny, const T *fP, T rho0,
                                          T *fb) {
    T dr, r, u, v;
    moments(fP, rho0, dr, r, u, v);
    const T bvl[5] = {bv3[0], bv3[1], bv3[2], T(0), T(0)};
    boundary_values(type, bvl, 0, 1, snx, sny, fP, dr, r, u, v, rho0, fb);
}

// lf += (d fb / d fP)^T c and lb3 += (d fb / d(rho_b, u_b, v_b))^T c for one boundary face.
__device__ __forceinline__ void adj_bvals_T(int type, const double *bv3, double snx, double sny,
                                            const double *fP, double rho0, const double *c,
                                            double *lf, double *lb3) {
    for (int k = 0; k < kQ + 3; ++k) {
        Dual fd[kQ], bd[3], fb[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) fd[a] = Dual(fP[a], k == a ? 1.0 : 0.0);
#pragma unroll
        for (int q = 0; q < 3; ++q) bd[q] = Dual(bv3[q], k == kQ + q ? 1.0 : 0.0);
        adj_bvals<Dual>(type, bd, Dual(snx), Dual(sny), fd, Dual(rho0), fb);
        double s = 0;
#pragma unroll
        for (int a = 0; a < kQ; ++a) s += fb[a].d * c[a];
        if (k < kQ)
            lf[k] += s;
        else if (lb3 != nullptr)
            lb3[k - kQ] += s;
    }
}

// acc of cell i (the forward flux sum) from a stage value and its gradient.
__device__ __forceinline__ void adj_flux_acc(int i, const double *fs, const double *g, const Geo<double> &G,
                                             double rho0, double *acc) {
    const size_t np = G.np;
    double fi[kQ];
    load9(fs, np, i, fi);
#pragma unroll
    for (int a = 0; a < kQ; ++a) acc[a] = 0.0;
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + i];
        if (nb == kNone) continue;
        const double snx = G.sn[(2 * m) * np + i], sny = G.sn[(2 * m + 1) * np + i];
        if (nb >= 0) {
            const double rox = G.rown[(2 * m) * np + i], roy = G.rown[(2 * m + 1) * np + i];
            const double rnx = G.rnbr[(2 * m) * np + i], rny = G.rnbr[(2 * m + 1) * np + i];
#pragma unroll
            for (int a = 0; a < kQ; ++a) {
                const double en = edot<double>(a, snx, sny);
                double fv;
                if (en >= 0.0)
                    fv = fi[a] + g[(2 * a) * np + i] * rox + g[(2 * a + 1) * np + i] * roy;
                else
                    fv = fs[a * np + nb] + g[(2 * a) * np + nb] * rnx + g[(2 * a + 1) * np + nb] * rny;
                acc[a] += en * fv;
            }
        } else {
            const int b = -nb - 1;
            double dr, r, u, v, fb[kQ];
            moments(fi, rho0, dr, r, u, v);
            boundary_values(G.btype[b], G.bval + b, 0, G.nbt, snx, sny, fi, dr, r, u, v, rho0, fb);
#pragma unroll
            for (int a = 0; a < kQ; ++a) acc[a] += edot<double>(a, snx, sny) * fb[a];
        }
    }
}

__device__ __forceinline__ void adj_bv3(const Geo<double> &G, int b, double *bv3) {
    for (int q = 0; q < 3; ++q) bv3[q] = G.bval[q * G.nbt + b];
}

// ---- transposed flux: la (adjoint of acc) -> lf += (d acc / d f)^T la, lg = (d acc / d g)^T la
__global__ void __launch_bounds__(kTile) k_adj_fluxT(const double *__restrict__ fs, const double *__restrict__ la,
                                                     double *__restrict__ lf, double *__restrict__ lg,
                                                     double *__restrict__ lbval, Geo<double> G,
                                                     const int *__restrict__ back) {
    const int j = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const double rho0 = G.ip[G.tile_inst[blockIdx.x]].rho0;
    double lfj[kQ], lgx[kQ], lgy[kQ], laj[kQ], fj[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lfj[a] = lf[a * np + j];
        lgx[a] = lgy[a] = 0.0;
        laj[a] = la[a * np + j];
        fj[a] = fs[a * np + j];
    }
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + j];
        if (nb == kNone) continue;
        const double snx = G.sn[(2 * m) * np + j], sny = G.sn[(2 * m + 1) * np + j];
        if (nb >= 0) {
            const double rox = G.rown[(2 * m) * np + j], roy = G.rown[(2 * m + 1) * np + j];
            const int b = back[m * np + j];
            const double six = G.sn[(2 * b) * np + nb], siy = G.sn[(2 * b + 1) * np + nb];
            const double rix = G.rnbr[(2 * b) * np + nb], riy = G.rnbr[(2 * b + 1) * np + nb];
#pragma unroll
            for (int a = 1; a < kQ; ++a) {
                const double en = edot<double>(a, snx, sny);
                if (en >= 0.0) {  // this cell's own flux took its own reconstruction
                    lfj[a] += en * laj[a];
                    lgx[a] += en * rox * laj[a];
                    lgy[a] += en * roy * laj[a];
                }
                const double eni = edot<double>(a, six, siy);
                if (!(eni >= 0.0)) {  // the neighbour's flux through this face took this cell's
                    const double lai = la[a * np + nb];
                    lfj[a] += eni * lai;
                    lgx[a] += eni * rix * lai;
                    lgy[a] += eni * riy * lai;
                }
            }
        } else {
            const int bf = -nb - 1;
            double c[kQ], bv3[3];
#pragma unroll
            for (int a = 0; a < kQ; ++a) c[a] = edot<double>(a, snx, sny) * laj[a];
            adj_bv3(G, bf, bv3);
            double lb3[3] = {0, 0, 0};
            adj_bvals_T(G.btype[bf], bv3, snx, sny, fj, rho0, c, lfj, lb3);
            if (lbval != nullptr)
                for (int q = 0; q < 3; ++q) lbval[q * G.nbt + bf] += lb3[q];
        }
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lf[a * np + j] = lfj[a];
        lg[(2 * a) * np + j] = lgx[a];
        lg[(2 * a + 1) * np + j] = lgy[a];
    }
}

// ---- transposed gradient: lf += (d g / d f)^T lg
__global__ void __launch_bounds__(kTile) k_adj_gradT(const double *__restrict__ fs, const double *__restrict__ lg,
                                                     double *__restrict__ lf, double *__restrict__ lbval,
                                                     Geo<double> G, const int *__restrict__ back) {
    const int j = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const double rho0 = G.ip[G.tile_inst[blockIdx.x]].rho0;
    double lfj[kQ], lgx[kQ], lgy[kQ], fj[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lfj[a] = lf[a * np + j];
        lgx[a] = lg[(2 * a) * np + j];
        lgy[a] = lg[(2 * a + 1) * np + j];
        fj[a] = fs[a * np + j];
    }
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + j];
        if (nb == kNone) continue;
        const double wx = G.lsq[(2 * m) * np + j], wy = G.lsq[(2 * m + 1) * np + j];
        double c[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            c[a] = wx * lgx[a] + wy * lgy[a];
            lfj[a] -= c[a];  // g_j = sum_m W_m (f_m - f_j)
        }
        if (nb >= 0) {
            const int b = back[m * np + j];
            const double wix = G.lsq[(2 * b) * np + nb], wiy = G.lsq[(2 * b + 1) * np + nb];
#pragma unroll
            for (int a = 0; a < kQ; ++a)
                lfj[a] += wix * lg[(2 * a) * np + nb] + wiy * lg[(2 * a + 1) * np + nb];
        } else {
            const int bf = -nb - 1;
            double bv3[3], lb3[3] = {0, 0, 0};
            adj_bv3(G, bf, bv3);
            adj_bvals_T(G.btype[bf], bv3, G.sn[(2 * m) * np + j], G.sn[(2 * m + 1) * np + j], fj, rho0, c,
                        lfj, lb3);
            if (lbval != nullptr)
                for (int q = 0; q < 3; ++q) lbval[q * G.nbt + bf] += lb3[q];
        }
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) lf[a * np + j] = lfj[a];
}

// ---- adjoints of the geometry arrays read by one flux and gradient evaluation: with la the
// adjoint of acc and lg that of g at this stage value, accumulate dJ/d(sn, rown, rnbr, lsq) of
// every face slot of the cell (one thread per cell, its own slots only).
__global__ void __launch_bounds__(kTile) k_adj_geom(const double *__restrict__ fs, const double *__restrict__ g,
                                                    const double *__restrict__ la, const double *__restrict__ lg,
                                                    Geo<double> G, double *__restrict__ a_sn,
                                                    double *__restrict__ a_lsq, double *__restrict__ a_rown,
                                                    double *__restrict__ a_rnbr) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const double rho0 = G.ip[G.tile_inst[blockIdx.x]].rho0;
    double fi[kQ];
    load9(fs, np, i, fi);
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + i];
        if (nb == kNone) continue;
        const double snx = G.sn[(2 * m) * np + i], sny = G.sn[(2 * m + 1) * np + i];
        double s_snx = 0, s_sny = 0, s_rox = 0, s_roy = 0, s_rnx = 0, s_rny = 0, s_lx = 0, s_ly = 0;
        if (nb >= 0) {
            const double rox = G.rown[(2 * m) * np + i], roy = G.rown[(2 * m + 1) * np + i];
            const double rnx = G.rnbr[(2 * m) * np + i], rny = G.rnbr[(2 * m + 1) * np + i];
#pragma unroll
            for (int a = 0; a < kQ; ++a) {
                const double en = edot<double>(a, snx, sny);
                const double l = la[a * np + i];
                const double fm = fs[a * np + nb];
                double fv;
                if (en >= 0.0) {
                    const double gx = g[(2 * a) * np + i], gy = g[(2 * a + 1) * np + i];
                    fv = fi[a] + gx * rox + gy * roy;
                    s_rox += l * en * gx;
                    s_roy += l * en * gy;
                } else {
                    const double gx = g[(2 * a) * np + nb], gy = g[(2 * a + 1) * np + nb];
                    fv = fm + gx * rnx + gy * rny;
                    s_rnx += l * en * gx;
                    s_rny += l * en * gy;
                }
                s_snx += l * ex_of(a) * fv;
                s_sny += l * ey_of(a) * fv;
                s_lx += lg[(2 * a) * np + i] * (fm - fi[a]);
                s_ly += lg[(2 * a + 1) * np + i] * (fm - fi[a]);
            }
        } else {
            const int bf = -nb - 1;
            double dr, r, u, v, fb[kQ];
            moments(fi, rho0, dr, r, u, v);
            boundary_values(G.btype[bf], G.bval + bf, 0, G.nbt, snx, sny, fi, dr, r, u, v, rho0, fb);
#pragma unroll
            for (int a = 0; a < kQ; ++a) {
                const double l = la[a * np + i];
                s_snx += l * ex_of(a) * fb[a];
                s_sny += l * ey_of(a) * fb[a];
                s_lx += lg[(2 * a) * np + i] * (fb[a] - fi[a]);
                s_ly += lg[(2 * a + 1) * np + i] * (fb[a] - fi[a]);
            }
        }
        a_sn[(2 * m) * np + i] += s_snx;
        a_sn[(2 * m + 1) * np + i] += s_sny;
        a_lsq[(2 * m) * np + i] += s_lx;
        a_lsq[(2 * m + 1) * np + i] += s_ly;
        a_rown[(2 * m) * np + i] += s_rox;
        a_rown[(2 * m + 1) * np + i] += s_roy;
        a_rnbr[(2 * m) * np + i] += s_rnx;
        a_rnbr[(2 * m + 1) * np + i] += s_rny;
    }
}

// ---- stage 3: lf3 = L, lc = L, la3 = -dt/3 L
__global__ void __launch_bounds__(kTile) k_adj_stage3(const double *__restrict__ L, double *__restrict__ lf3,
                                                      double *__restrict__ lc, double *__restrict__ la,
                                                      Geo<double> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const double dt = G.ip[G.tile_inst[blockIdx.x]].dt;
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        const double l = L[a * np + i];
        lf3[a * np + i] = l;
        lc[a * np + i] = l;
        la[a * np + i] = -(dt * (1.0 / 3.0)) * l;
    }
}

// ---- stage 2: from lf3, lc -> lB, la2 (X = B - dt/2 a2, f3 = S2(X), C' = C + dt/6 a2)
__global__ void __launch_bounds__(kTile) k_adj_stage2(const double *__restrict__ Bv, const double *__restrict__ f2,
                                                      const double *__restrict__ g2, const double *__restrict__ tau,
                                                      const double *__restrict__ lf3, const double *__restrict__ lc,
                                                      double *__restrict__ lB, double *__restrict__ la,
                                                      Geo<double> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    const double dt = P.dt;
    double acc[kQ], X[kQ], l3[kQ];
    adj_flux_acc(i, f2, g2, G, P.rho0, acc);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        X[a] = Bv[a * np + i] - 0.5 * dt * acc[a];
        l3[a] = lf3[a * np + i];
    }
    double lX[kQ];
    for (int k = 0; k < kQ; ++k) {
        Dual xd[kQ], f3[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) xd[a] = Dual(X[a], k == a ? 1.0 : 0.0);
        adj_stage2<Dual>(xd, Dual(P.rho0), Dual(dt), Dual(tau[i]), f3);
        double s = 0;
#pragma unroll
        for (int a = 0; a < kQ; ++a) s += f3[a].d * l3[a];
        lX[k] = s;
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lB[a * np + i] = lX[a];
        la[a * np + i] = -0.5 * dt * lX[a] + dt * (1.0 / 6.0) * lc[a * np + i];
    }
}

// ---- stage 1: from lf2, lB, lc -> lf0 (=), la1 ((f2, B, C) = S1(f0, a1))
__global__ void __launch_bounds__(kTile) k_adj_stage1(const double *__restrict__ f0, const double *__restrict__ s1,
                                                      const double *__restrict__ g1, const double *__restrict__ tau,
                                                      const double *__restrict__ lf2, const double *__restrict__ lB,
                                                      const double *__restrict__ lc, double *__restrict__ lf0,
                                                      double *__restrict__ la, Geo<double> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    double acc[kQ], x0[kQ], l2[kQ], lb[kQ], lcc[kQ];
    adj_flux_acc(i, s1, g1, G, P.rho0, acc);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        x0[a] = f0[a * np + i];
        l2[a] = lf2[a * np + i];
        lb[a] = lB[a * np + i];
        lcc[a] = lc[a * np + i];
    }
    for (int k = 0; k < 2 * kQ; ++k) {
        Dual fd[kQ], ad[kQ], f2[kQ], B[kQ], C[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            fd[a] = Dual(x0[a], k == a ? 1.0 : 0.0);
            ad[a] = Dual(acc[a], k == kQ + a ? 1.0 : 0.0);
        }
        adj_stage1<Dual>(fd, ad, Dual(P.rho0), Dual(P.dt), Dual(tau[i]), f2, B, C);
        double s = 0;
#pragma unroll
        for (int a = 0; a < kQ; ++a) s += f2[a].d * l2[a] + B[a].d * lb[a] + C[a].d * lcc[a];
        if (k < kQ)
            lf0[k * np + i] = s;
        else
            la[(k - kQ) * np + i] = s;
    }
}

// ---- relaxation of stage 1: lf0 += (d s1 / d f0)^T ls1
__global__ void __launch_bounds__(kTile) k_adj_relax(const double *__restrict__ f0, const double *__restrict__ tau,
                                                     const double *__restrict__ ls1, double *__restrict__ lf0,
                                                     Geo<double> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    double x0[kQ], l1[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        x0[a] = f0[a * np + i];
        l1[a] = ls1[a * np + i];
    }
    for (int k = 0; k < kQ; ++k) {
        Dual fd[kQ], s1[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) fd[a] = Dual(x0[a], k == a ? 1.0 : 0.0);
        adj_relax<Dual>(fd, Dual(P.rho0), Dual(P.dt), Dual(tau[i]), s1);
        double s = 0;
#pragma unroll
        for (int a = 0; a < kQ; ++a) s += s1[a].d * l1[a];
        lf0[k * np + i] += s;
    }
}

// ---- objective J = (cx Fx + cy Fy) / (q l) over the wall faces of one instance: its
// derivative with respect to f (into L, which is zeroed first) and to the boundary values
__global__ void __launch_bounds__(kTile) k_adj_seed(const double *__restrict__ fn, const double *__restrict__ bnrm,
                                                    const double *__restrict__ blen, int inst, double cx, double cy,
                                                    double *__restrict__ L, double *__restrict__ lbval,
                                                    double *__restrict__ a_bnrm, double *__restrict__ a_blen,
                                                    Geo<double> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const double rho0 = G.ip[G.tile_inst[blockIdx.x]].rho0;
    double lfi[kQ], fi[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lfi[a] = 0.0;
        fi[a] = fn[a * np + i];
    }
    if (G.tile_inst[blockIdx.x] == inst) {
        for (int m = 0; m < 4; ++m) {
            const int nb = G.nbr[m * np + i];
            if (nb == kNone || nb >= 0) continue;
            const int bf = -nb - 1;
            if (G.btype[bf] != FVLBM_BC_WALL) continue;
            const double nx = bnrm[bf], ny = bnrm[G.nbt + bf];
            double c[kQ], bv3[3], lb3[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < kQ; ++a)
                c[a] = edot<double>(a, nx, ny) * blen[bf] * (ex_of(a) * cx + ey_of(a) * cy);
            adj_bv3(G, bf, bv3);
            adj_bvals_T(FVLBM_BC_WALL, bv3, nx, ny, fi, rho0, c, lfi, lb3);
            if (lbval != nullptr)
                for (int q = 0; q < 3; ++q) lbval[q * G.nbt + bf] += lb3[q];
            if (a_bnrm != nullptr) {  // F = sum_a e_a (e_a . n) (f_bc + w rho0) dl
                double dr, r, u, v, fb[kQ], sx = 0, sy = 0, sl = 0;
                moments(fi, rho0, dr, r, u, v);
                boundary_values(FVLBM_BC_WALL, G.bval + bf, 0, G.nbt, nx, ny, fi, dr, r, u, v, rho0, fb);
                for (int a = 0; a < kQ; ++a) {
                    const double wgt = (ex_of(a) * cx + ey_of(a) * cy) * (fb[a] + w_of<double>(a) * rho0);
                    sx += wgt * ex_of(a);
                    sy += wgt * ey_of(a);
                    sl += wgt * edot<double>(a, nx, ny);
                }
                a_bnrm[bf] = sx * blen[bf];
                a_bnrm[G.nbt + bf] = sy * blen[bf];
                a_blen[bf] = sl;
            }
        }
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) L[a * np + i] = lfi[a];
}

// out[perm[k] * 9 + a] = L[a][off + k] (no offset: an adjoint, not a distribution)
__global__ void k_adj_gather(const double *__restrict__ L, const int *__restrict__ perm, int off, int nc,
                             size_t np, double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const int dst = perm[k];
    for (int a = 0; a < kQ; ++a) out[static_cast<size_t>(dst) * kQ + a] = L[a * np + off + k];
}

}  // namespace fvlbm

namespace {

// Device buffers of one adjoint call, freed when it returns.
struct AdjScratch {
    std::vector<void *> p;
    size_t bytes = 0;
    ~AdjScratch() {
        for (void *x : p) cudaFree(x);
    }
    double *get(size_t n, cudaError_t *err) {
        void *x = nullptr;
        const size_t b = std::max<size_t>(n, 2) * sizeof(double);
        const cudaError_t e = cudaMalloc(&x, b);
        if (e != cudaSuccess) {
            if (*err == cudaSuccess) *err = e;
            return nullptr;
        }
        p.push_back(x);
        bytes += b;
        return static_cast<double *>(x);
    }
};

// Stage values of one step that its adjoint reads.
struct AdjStep {
    double *s1, *g1, *f2, *g2, *B, *C, *f3, *g3, *mac;
};

// One two-pass FP64 step f_in -> f_out (the launches of the laminar two-pass path, with the
// stage values kept in S).
void adj_forward_step(fvlbm_handle *h, const Geo<double> &G, const double *f_in, double *f_out,
                      const AdjStep &S) {
    const dim3 grid(h->ntiles), block(kTile);
    cudaStream_t s = h->stream;
    const double *tau = static_cast<const double *>(h->tau);
    double *fin = const_cast<double *>(f_in);
    k_stage1<double><<<grid, block, 0, s>>>(f_in, S.s1, tau, G);
    k_grad<double, false><<<grid, block, 0, s>>>(S.s1, S.g1, G);
    k_flux_stage<double, 1, false><<<grid, block, 0, s>>>(S.s1, S.g1, S.f2, fin, S.B, S.C, tau, S.mac,
                                                          nullptr, G);
    k_grad<double, false><<<grid, block, 0, s>>>(S.f2, S.g2, G);
    k_flux_stage<double, 2, false><<<grid, block, 0, s>>>(S.f2, S.g2, S.f3, fin, S.B, S.C, tau, S.mac,
                                                          nullptr, G);
    k_grad<double, false><<<grid, block, 0, s>>>(S.f3, S.g3, G);
    k_flux_stage<double, 3, false><<<grid, block, 0, s>>>(S.f3, S.g3, nullptr, f_out, S.B, S.C, tau,
                                                          S.mac, nullptr, G);
}

// Adjoint of the step whose stage values S were just recomputed from f0: L (adjoint of f^{n+1})
// is replaced by the adjoint of f^n; boundary-value adjoints are added into lbval.
struct AdjVars {
    double *L, *lf3, *lc, *la, *lg, *lB, *lf2, *ls1, *lf0, *lbval;
    double *a_sn = nullptr, *a_lsq = nullptr, *a_rown = nullptr, *a_rnbr = nullptr;  // shape adjoint
    double *a_bnrm = nullptr, *a_blen = nullptr;
};

void adj_backward_step(fvlbm_handle *h, const Geo<double> &G, const double *f0, const AdjStep &S,
                       AdjVars &A) {
    const dim3 grid(h->ntiles), block(kTile);
    cudaStream_t s = h->stream;
    const size_t nq = static_cast<size_t>(kQ) * h->np;
    const double *tau = static_cast<const double *>(h->tau);
    const int *back = h->d_back;
    auto geom = [&](const double *fs, const double *g) {
        if (A.a_sn)
            k_adj_geom<<<grid, block, 0, s>>>(fs, g, A.la, A.lg, G, A.a_sn, A.a_lsq, A.a_rown, A.a_rnbr);
    };
    k_adj_stage3<<<grid, block, 0, s>>>(A.L, A.lf3, A.lc, A.la, G);
    k_adj_fluxT<<<grid, block, 0, s>>>(S.f3, A.la, A.lf3, A.lg, A.lbval, G, back);
    geom(S.f3, S.g3);
    k_adj_gradT<<<grid, block, 0, s>>>(S.f3, A.lg, A.lf3, A.lbval, G, back);
    k_adj_stage2<<<grid, block, 0, s>>>(S.B, S.f2, S.g2, tau, A.lf3, A.lc, A.lB, A.la, G);
    cudaMemsetAsync(A.lf2, 0, nq * sizeof(double), s);
    k_adj_fluxT<<<grid, block, 0, s>>>(S.f2, A.la, A.lf2, A.lg, A.lbval, G, back);
    geom(S.f2, S.g2);
    k_adj_gradT<<<grid, block, 0, s>>>(S.f2, A.lg, A.lf2, A.lbval, G, back);
    k_adj_stage1<<<grid, block, 0, s>>>(f0, S.s1, S.g1, tau, A.lf2, A.lB, A.lc, A.lf0, A.la, G);
    cudaMemsetAsync(A.ls1, 0, nq * sizeof(double), s);
    k_adj_fluxT<<<grid, block, 0, s>>>(S.s1, A.la, A.ls1, A.lg, A.lbval, G, back);
    geom(S.s1, S.g1);
    k_adj_gradT<<<grid, block, 0, s>>>(S.s1, A.lg, A.ls1, A.lbval, G, back);
    k_adj_relax<<<grid, block, 0, s>>>(f0, tau, A.ls1, A.lf0, G);
    std::swap(A.L, A.lf0);
}

int adjoint_impl(fvlbm_handle *h, int instance, int n_steps, const double *w, double *J, double *dJ_df,
                 double *dJ_dbedge, double *dJ_dxy) {
    if (!h || instance < 0 || instance >= h->ninst || n_steps < 0 || !w) return FVLBM_ERR_BAD_PARAM;
    if (h->precision != FVLBM_FP64 || h->sst || h->scheme != 0 || h->dtc != nullptr || h->limit_f ||
        h->per_stage || h->d_back == nullptr)
        return FVLBM_ERR_NOT_SUPPORTED;
    const InstInfo &I = h->inst[instance];
    if (dJ_dxy && (!I.mesh || !I.mesh->ppairs.empty())) return FVLBM_ERR_NOT_SUPPORTED;
    CK(cudaSetDevice(h->device));
    const Geo<double> G = geo_of<double>(h);
    const size_t np = h->np, nq = static_cast<size_t>(kQ) * np;
    const int K = std::max(1, static_cast<int>(std::ceil(std::sqrt(static_cast<double>(n_steps)))));
    const int nck = (n_steps + K - 1) / K;  // f^n kept at n = 0, K, 2K, ...
    cudaError_t err = cudaSuccess;
    AdjScratch M;
    std::vector<double *> ck(std::max(nck, 1)), seg(K);
    for (auto &x : ck) x = M.get(nq, &err);
    for (auto &x : seg) x = M.get(nq, &err);
    double *xa = M.get(nq, &err), *xb = M.get(nq, &err);
    AdjStep S{M.get(nq, &err), M.get(2 * nq, &err), M.get(nq, &err), M.get(2 * nq, &err), M.get(nq, &err),
              M.get(nq, &err), M.get(nq, &err), M.get(2 * nq, &err), M.get(3 * np, &err)};
    AdjVars A{M.get(nq, &err), M.get(nq, &err), M.get(nq, &err), M.get(nq, &err), M.get(2 * nq, &err),
              M.get(nq, &err), M.get(nq, &err), M.get(nq, &err), M.get(nq, &err),
              M.get(3 * static_cast<size_t>(std::max(h->nbt, 1)), &err)};
    const size_t nbt = std::max(h->nbt, 1);
    if (dJ_dxy) {
        A.a_sn = M.get(8 * np, &err);
        A.a_lsq = M.get(8 * np, &err);
        A.a_rown = M.get(8 * np, &err);
        A.a_rnbr = M.get(8 * np, &err);
        A.a_bnrm = M.get(2 * nbt, &err);
        A.a_blen = M.get(nbt, &err);
    }
    if (err != cudaSuccess) return cuda_fail(err);
    cudaStream_t s = h->stream;
    if (dJ_dxy) {
        for (double *x : {A.a_sn, A.a_lsq, A.a_rown, A.a_rnbr})
            CK(cudaMemsetAsync(x, 0, 8 * np * sizeof(double), s));
        CK(cudaMemsetAsync(A.a_bnrm, 0, 2 * nbt * sizeof(double), s));
        CK(cudaMemsetAsync(A.a_blen, 0, nbt * sizeof(double), s));
    }
    // forward sweep: f^N and the checkpoints
    CK(cudaMemcpyAsync(xa, h->fn, nq * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (nck > 0) CK(cudaMemcpyAsync(ck[0], xa, nq * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int n = 0; n < n_steps; ++n) {
        adj_forward_step(h, G, xa, xb, S);
        std::swap(xa, xb);
        if ((n + 1) % K == 0 && (n + 1) / K < nck)
            CK(cudaMemcpyAsync(ck[(n + 1) / K], xa, nq * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaGetLastError());
    // J at f^N and its direct derivatives
    double out[4];
    int rc = forces_impl(h, instance, 0.0, out, nullptr, nullptr, xa);
    if (rc) return rc;
    if (J) *J = w[0] * out[2] + w[1] * out[3];
    const double q = 0.5 * I.rho0 * I.uref * I.uref * I.lref;
    const double al = I.alpha_deg * M_PI / 180.0, ca = std::cos(al), sa = std::sin(al);
    const double cx = (w[0] * ca - w[1] * sa) / q, cy = (w[0] * sa + w[1] * ca) / q;
    CK(cudaMemsetAsync(A.lbval, 0, 3 * static_cast<size_t>(std::max(h->nbt, 1)) * sizeof(double), s));
    k_adj_seed<<<h->ntiles, kTile, 0, s>>>(xa, static_cast<const double *>(h->bnrm),
                                           static_cast<const double *>(h->blen), instance, cx, cy, A.L,
                                           A.lbval, A.a_bnrm, A.a_blen, G);
    CK(cudaGetLastError());
    // backward sweep, one checkpoint segment at a time
    for (int c = nck - 1; c >= 0; --c) {
        const int k0 = c * K, k1 = std::min(n_steps, k0 + K);
        CK(cudaMemcpyAsync(seg[0], ck[c], nq * sizeof(double), cudaMemcpyDeviceToDevice, s));
        for (int n = k0; n + 1 < k1; ++n) adj_forward_step(h, G, seg[n - k0], seg[n - k0 + 1], S);
        for (int n = k1 - 1; n >= k0; --n) {
            adj_forward_step(h, G, seg[n - k0], xb, S);
            adj_backward_step(h, G, seg[n - k0], S, A);
        }
        CK(cudaGetLastError());
    }
    if (dJ_df && I.nc > 0) {
        k_adj_gather<<<(I.nc + 255) / 256, 256, 0, s>>>(A.L, h->d_perm + perm_offset(h, instance), I.cell_off,
                                                         I.nc, np, xb);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(dJ_df, xb, sizeof(double) * kQ * static_cast<size_t>(I.nc), cudaMemcpyDeviceToHost,
                           s));
    }
    std::vector<double> lb(3 * static_cast<size_t>(std::max(I.nb, 1)));
    if (dJ_dbedge && I.nb > 0)
        for (int c = 0; c < 3; ++c)
            CK(cudaMemcpyAsync(lb.data() + static_cast<size_t>(c) * I.nb,
                               A.lbval + static_cast<size_t>(c) * h->nbt + I.bface_off, sizeof(double) * I.nb,
                               cudaMemcpyDeviceToHost, s));
    // shape adjoint: the instance's slices of the geometry adjoints, in input order, then the
    // reverse of the host preprocessing
    GeometryAdjoint GA;
    std::vector<int> perm(std::max(I.nc, 1));
    std::vector<double> runs;
    if (dJ_dxy) {
        const size_t nc = I.nc;
        CK(cudaMemcpyAsync(perm.data(), h->d_perm + perm_offset(h, instance), sizeof(int) * nc,
                           cudaMemcpyDeviceToHost, s));
        runs.resize(4 * 8 * nc + 3 * static_cast<size_t>(std::max(I.nb, 1)));
        const double *src[4] = {A.a_sn, A.a_lsq, A.a_rown, A.a_rnbr};
        for (int q = 0; q < 4; ++q)
            for (int c = 0; c < 8; ++c)
                CK(cudaMemcpyAsync(runs.data() + (8 * q + c) * nc, src[q] + c * np + I.cell_off, sizeof(double) * nc,
                                   cudaMemcpyDeviceToHost, s));
        double *bt = runs.data() + 32 * nc;
        if (I.nb > 0) {
            CK(cudaMemcpyAsync(bt, A.a_bnrm + I.bface_off, sizeof(double) * I.nb, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(bt + I.nb, A.a_bnrm + h->nbt + I.bface_off, sizeof(double) * I.nb,
                               cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(bt + 2 * I.nb, A.a_blen + I.bface_off, sizeof(double) * I.nb, cudaMemcpyDeviceToHost,
                               s));
        }
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    if (dJ_dxy) {
        const size_t nc = I.nc;
        const MeshCopy &mc = *I.mesh;
        std::vector<double> *dst[4] = {&GA.sn, &GA.lsq, &GA.rown, &GA.rnbr};
        for (int q = 0; q < 4; ++q) {
            dst[q]->assign(8 * nc, 0.0);
            for (size_t k = 0; k < nc; ++k)
                for (int c = 0; c < 8; ++c)  // component c = 2 l + (x, y) of slot l
                    (*dst[q])[8 * static_cast<size_t>(perm[k]) + c] = runs[(8 * q + c) * nc + k];
        }
        const size_t nbe = mc.btype.size();
        GA.bnrm.assign(2 * nbe, 0.0);
        GA.blen.assign(nbe, 0.0);
        const double *bt = runs.data() + 32 * nc;
        for (int f = 0; f < I.nb; ++f) {
            const int e = I.bedge_of[f];
            GA.bnrm[2 * e] = bt[f];
            GA.bnrm[2 * e + 1] = bt[I.nb + f];
            GA.blen[e] = bt[2 * I.nb + f];
        }
        const fvlbm_mesh Mm{I.n_nodes, mc.xy.data(), I.nc, mc.cell_ptr.data(), mc.cell_nodes.data()};
        const fvlbm_bc Bm{static_cast<int>(nbe), mc.bnodes.data(), mc.btype.data(), mc.bval.data(), 0, nullptr,
                          nullptr};
        std::string why;
        const int grc = geometry_adjoint(Mm, Bm, GA, dJ_dxy, &why);
        if (grc) return grc;
    }
    if (dJ_dbedge) {
        std::fill(dJ_dbedge, dJ_dbedge + 5 * static_cast<size_t>(I.n_bedges_in), 0.0);
        for (int b = 0; b < I.nb; ++b)
            for (int c = 0; c < 3; ++c)
                dJ_dbedge[5 * static_cast<size_t>(I.bedge_of[b]) + c] = lb[static_cast<size_t>(c) * I.nb + b];
    }
    return FVLBM_OK;
}

}  // namespace
