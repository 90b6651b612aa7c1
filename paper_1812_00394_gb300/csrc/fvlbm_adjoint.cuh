// fvlbm_adjoint.cuh -- discrete adjoint (reverse mode) of the FP64 time step, included into
// fvlbm_kernels.cu after the handle and its helpers.
//
// The map differentiated is the two-pass IMEX step exactly as the library runs it (Sec. 3.2,
// Steps 1-7): on SST instances the k-omega SST solve first (its reverse is in
// fvlbm_adjoint_sst.cuh), then f^(1) = R(f^n) (Eq. (fnewstage), J = 1), three gradient + flux
// evaluations (Step 2, Eq. (advection)) and the stage algebra of the two accumulators.  Per step
//   s1 = R(f0);  a1 = A(s1);  (f2, B, C) = S1(f0, a1);  a2 = A(f2);  f3 = S2(B - dt/2 a2);
//   C' = C + dt/6 a2;  a3 = A(f3);  f^{n+1} = f3 + C' - dt/3 a3,
// with A(f) = sum over faces of (e . n dl / A) times the upwind linear face value built from
// the least-squares gradient, boundary faces taking the boundary values of Part I, and R, S1,
// S2 relaxing with the step's tau.  The adjoint runs these in reverse: the linear flux and
// gradient operators are transposed by gathering over each cell's faces (the neighbour's view
// of a shared face comes from its back slot); the per-cell maps R, S1, S2 and the boundary
// values are transposed in closed form (they are affine but for f^eq, whose transposed Jacobian
// is written out below).  The explicit Euler comparison scheme and the per-stage SST reading
// have their own forward recompute and reverse (adj_forward_step, adj_backward_step).  Stage
// values stay in device memory for whole runs of steps, and longer runs are reversed on a
// binomial checkpoint schedule (see adjoint_impl).

namespace fvlbm {

// ---- per-cell maps.  Each is affine in its inputs except through the equilibrium of a stage
// value X, f^eq(X) = feq_dev(moments(X)), so its adjoint needs only the transposed Jacobian of
// that map, formed in closed form:
//   f^eq_a = w_a [drho + rho P_a],  P_a = 3 e_a.u + 4.5 (e_a.u)^2 - 1.5 u.u,  u = j / rho,
//   dP_a/du = (3 + 9 e_a.u) e_a - 3 u,  du/dj = 1/rho,  du/drho = -u/rho,
// and lam_b += l_drho + e_b . l_j for the moments drho = sum d, j = sum e d.
// For f^eq_a = w_a [d + r P_a(u, v)] with d and r moving together (d r = d d): the adjoints
// l_d = sum_a mu_a w_a (1 + P_a) and l_(u, v) = sum_a mu_a w_a r dP_a/d(u, v).
__device__ __forceinline__ void feq_uv_vjp(double r, double u, double v, const double *mu, double &l_d,
                                           double &l_u, double &l_v) {
    const double uu = 1.5 * (u * u + v * v);
    l_d = l_u = l_v = 0.0;
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        const double eu = edot<double>(a, u, v);
        const double wm = w_of<double>(a) * mu[a];
        l_d += wm * (1.0 + 3.0 * eu + 4.5 * eu * eu - uu);
        const double c = wm * r * (3.0 + 9.0 * eu);
        l_u += c * ex_of(a) - 3.0 * wm * r * u;
        l_v += c * ey_of(a) - 3.0 * wm * r * v;
    }
}

// lam += adjoint of the moments (drho, rho, u, v) of X given l_d (drho and rho together) and
// l_(u, v), with u = j / rho.
__device__ __forceinline__ void moments_vjp(double r, double u, double v, double l_d, double l_u, double l_v,
                                            double *lam) {
    const double ir = 1.0 / r;
    const double l_jx = l_u * ir, l_jy = l_v * ir;
    l_d -= (l_u * u + l_v * v) * ir;
#pragma unroll
    for (int a = 0; a < kQ; ++a) lam[a] += l_d + edot<double>(a, l_jx, l_jy);
}

// lam += (d f^eq(moments(X)) / d X)^T mu
__device__ __forceinline__ void feq_vjp(const double *X, double rho0, const double *mu, double *lam) {
    double dr, r, u, v, l_d, l_u, l_v;
    moments(X, rho0, dr, r, u, v);
    feq_uv_vjp(r, u, v, mu, l_d, l_u, l_v);
    moments_vjp(r, u, v, l_d, l_u, l_v, lam);
}

// lf += (d fb / d fP)^T c and lb3 += (d fb / d(rho_b, u_b, v_b))^T c for one boundary face whose
// values fb = boundary_values(type, ...) are formed from the owner's fP:
//   wall, inlet:  fb = fP + f^eq(drho_P, rho_P, u_b, v_b) - f^eq(moments(fP))
//   outlet:       fb = fP + f^eq(rho_b - rho0, rho_b, u_P, v_P) - f^eq(moments(fP))
//   far field:    fb_a = f^eq(rho_b - rho0, rho_b, u_b, v_b)_a where e_a . n < 0, else fP_a
__device__ __forceinline__ void adj_bvals_T(int type, const double *bv3, double snx, double sny,
                                            const double *fP, double rho0, const double *c,
                                            double *lf, double *lb3) {
    double dr, r, u, v, l_d, l_u, l_v;
    moments(fP, rho0, dr, r, u, v);
    const double rb = bv3[0], ub = bv3[1], vb = bv3[2];
    if (type == FVLBM_BC_WALL || type == FVLBM_BC_INLET || type == FVLBM_BC_OUTLET) {
        double mneg[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            lf[a] += c[a];
            mneg[a] = -c[a];
        }
        feq_vjp(fP, rho0, mneg, lf);
        if (type == FVLBM_BC_OUTLET) {  // f^eq at rho_b and the owner's velocity
            feq_uv_vjp(rb, u, v, c, l_d, l_u, l_v);
            moments_vjp(r, u, v, 0.0, l_u, l_v, lf);
            lb3[0] += l_d;
        } else {  // f^eq at the owner's density and the boundary velocity
            feq_uv_vjp(r, ub, vb, c, l_d, l_u, l_v);
#pragma unroll
            for (int a = 0; a < kQ; ++a) lf[a] += l_d;
            lb3[1] += l_u;
            lb3[2] += l_v;
        }
    } else {
        double cin[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            const bool in = edot<double>(a, snx, sny) < 0.0;
            cin[a] = in ? c[a] : 0.0;
            if (!in) lf[a] += c[a];
        }
        feq_uv_vjp(rb, ub, vb, cin, l_d, l_u, l_v);
        lb3[0] += l_d;
        lb3[1] += l_u;
        lb3[2] += l_v;
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

// ---- transposed flux over interior faces: la (adjoint of acc) -> lf += (d acc / d f)^T la,
// lg = (d acc / d g)^T la (boundary faces: k_adj_bndT)
__global__ void __launch_bounds__(kTile) k_adj_fluxT(const double *__restrict__ la, double *__restrict__ lf,
                                                     double *__restrict__ lg, Geo<double> G,
                                                     const int *__restrict__ back) {
    const int j = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    double lfj[kQ], lgx[kQ], lgy[kQ], laj[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lfj[a] = lf[a * np + j];
        lgx[a] = lgy[a] = 0.0;
        laj[a] = la[a * np + j];
    }
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + j];
        if (nb < 0) continue;  // no face, or a boundary face
        const double snx = G.sn[(2 * m) * np + j], sny = G.sn[(2 * m + 1) * np + j];
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
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lf[a * np + j] = lfj[a];
        lg[(2 * a) * np + j] = lgx[a];
        lg[(2 * a + 1) * np + j] = lgy[a];
    }
}

// ---- transposed gradient, linear part: lf += (d g / d f)^T lg with the boundary values held
// fixed (g_j = sum_m W_m (f_m - f_j)); their dependence on f_j is added by k_adj_bndT
__global__ void __launch_bounds__(kTile) k_adj_gradT(const double *__restrict__ lg, double *__restrict__ lf,
                                                     Geo<double> G, const int *__restrict__ back,
                                                     const double *__restrict__ lnb) {
    const int j = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    double lfj[kQ], lgx[kQ], lgy[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lfj[a] = lf[a * np + j];
        lgx[a] = lg[(2 * a) * np + j];
        lgy[a] = lg[(2 * a + 1) * np + j];
    }
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + j];
        if (nb == kNone) continue;
        const double wx = G.lsq[(2 * m) * np + j], wy = G.lsq[(2 * m + 1) * np + j];
#pragma unroll
        for (int a = 0; a < kQ; ++a) lfj[a] -= wx * lgx[a] + wy * lgy[a];
        if (nb >= 0) {
            const int b = back[m * np + j];
            const double wix = G.lsq[(2 * b) * np + nb], wiy = G.lsq[(2 * b + 1) * np + nb];
#pragma unroll
            for (int a = 0; a < kQ; ++a)
                lfj[a] += wix * lg[(2 * a) * np + nb] + wiy * lg[(2 * a + 1) * np + nb];
            if (lnb != nullptr)  // the neighbour's limiter took this cell's value as its extreme
                for (int a = 1; a < kQ; ++a) lfj[a] += lnb[(a * 4 + b) * np + nb];
        }
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) lf[a * np + j] = lfj[a];
}

// ---- limiter on grad f (reading variant 1): the stage used g = phi g_raw with the
// Venkatakrishnan factor phi = min over faces of r(d1, d2) (d2 = g_raw . r_m, d1 = the distance
// from f_i to the max / min over the cell, its neighbours and its boundary values; e2 = A^(3/2)).
// In: lg, the adjoint of the limited gradient.  Out: lg <- the adjoint of g_raw; lf_i gets the
// adjoint of f_i through d1; the extreme's share goes to the per-face buffers, lnb[(a * 4 + m)
// * np + i] for a neighbour (gathered by k_adj_gradT) and lbf for a boundary value (added by
// k_adj_bndT).  Branches (extremes, the minimum over faces) follow the values, ties keeping the
// first argument, as the forward's fmin / fmax.
__global__ void __launch_bounds__(kTile) k_adj_limT(const double *__restrict__ fs, double *__restrict__ lg,
                                                    double *__restrict__ lf, double *__restrict__ lnb,
                                                    double *__restrict__ lbf, Geo<double> G,
                                                    double *__restrict__ a_rown, double *__restrict__ a_area) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    for (int c = 0; c < 4 * kQ; ++c) {
        lnb[c * np + i] = 0.0;
        lbf[c * np + i] = 0.0;
    }
    if (!(P.variant & 1)) return;
    const double rho0 = P.rho0;
    double fi[kQ], fbv[4][kQ];
    load9(fs, np, i, fi);
    bool has[4];
    int nbs[4];
    for (int m = 0; m < 4; ++m) {
        nbs[m] = G.nbr[m * np + i];
        has[m] = nbs[m] != kNone;
        if (has[m] && nbs[m] < 0) {
            const int b = -nbs[m] - 1;
            double dr, r, u, v;
            moments(fi, rho0, dr, r, u, v);
            boundary_values(G.btype[b], G.bval + b, 0, G.nbt, G.sn[(2 * m) * np + i], G.sn[(2 * m + 1) * np + i],
                            fi, dr, r, u, v, rho0, fbv[m]);
        }
    }
    const double ar = G.area[i];
    const double e2 = ar * sqrt(ar);
    double lfi[kQ], l_e2 = 0.0;
#pragma unroll
    for (int a = 0; a < kQ; ++a) lfi[a] = lf[a * np + i];
    for (int a = 1; a < kQ; ++a) {
        // raw gradient and the extremes (index -1: the cell itself)
        double gx = 0.0, gy = 0.0, lo = fi[a], hi = fi[a];
        int ilo = -1, ihi = -1;
        for (int m = 0; m < 4; ++m) {
            if (!has[m]) continue;
            const double fm = nbs[m] >= 0 ? fs[a * np + nbs[m]] : fbv[m][a];
            const double d = fm - fi[a];
            gx += G.lsq[(2 * m) * np + i] * d;
            gy += G.lsq[(2 * m + 1) * np + i] * d;
            if (fm < lo) { lo = fm; ilo = m; }
            if (fm > hi) { hi = fm; ihi = m; }
        }
        double phi = 1.0, rsel_d1 = 0.0, rsel_d2 = 0.0;
        int msel = -1;
        bool upper = false;
        for (int m = 0; m < 4; ++m) {
            if (!has[m]) continue;
            const double d2 = gx * G.rown[(2 * m) * np + i] + gy * G.rown[(2 * m + 1) * np + i];
            if (d2 == 0.0) continue;
            const double d1 = d2 > 0.0 ? hi - fi[a] : lo - fi[a];
            const double r = ((d1 * d1 + e2) * d2 + 2.0 * d2 * d2 * d1) /
                             (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + e2) / d2;
            if (r < phi) {
                phi = r;
                msel = m;
                rsel_d1 = d1;
                rsel_d2 = d2;
                upper = d2 > 0.0;
            }
        }
        const double lgx = lg[(2 * a) * np + i], lgy = lg[(2 * a + 1) * np + i];
        const double l_phi = lgx * gx + lgy * gy;
        double lrx = phi * lgx, lry = phi * lgy;
        if (msel >= 0) {
            const double d1 = rsel_d1, d2 = rsel_d2;
            const double N = (d1 * d1 + e2) * d2 + 2.0 * d2 * d2 * d1;
            const double D = d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + e2;
            const double dr_d1 = ((2.0 * d1 * d2 + 2.0 * d2 * d2) * D - N * (2.0 * d1 + d2)) / (D * D * d2);
            const double dr_d2 = ((d1 * d1 + e2 + 4.0 * d2 * d1) * D * d2 - N * ((4.0 * d2 + d1) * d2 + D)) /
                                 (D * D * d2 * d2);
            const double l_d1 = l_phi * dr_d1, l_d2 = l_phi * dr_d2;
            lrx += l_d2 * G.rown[(2 * msel) * np + i];
            lry += l_d2 * G.rown[(2 * msel + 1) * np + i];
            if (a_rown != nullptr) {  // shape: d2 = g_raw . r_m, e2 = A^(3/2)
                a_rown[(2 * msel) * np + i] += l_d2 * gx;
                a_rown[(2 * msel + 1) * np + i] += l_d2 * gy;
                l_e2 += l_phi * (d2 * D - N) / (D * D * d2);
            }
            const int e = upper ? ihi : ilo;  // d1 = f_ext - f_i; the cell itself gives 0
            if (e >= 0) {
                lfi[a] -= l_d1;
                if (nbs[e] >= 0)
                    lnb[(a * 4 + e) * np + i] += l_d1;
                else
                    lbf[(a * 4 + e) * np + i] += l_d1;
            }
        }
        lg[(2 * a) * np + i] = lrx;
        lg[(2 * a + 1) * np + i] = lry;
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) lf[a * np + i] = lfi[a];
    if (a_area != nullptr) a_area[i] += l_e2 * 1.5 * sqrt(ar);
}

// ---- boundary faces: the face value f_bc(f_j, bval) enters the flux (weight e.n) and the
// gradient (weight W_m); one transposed local Jacobian per face serves both:
//   c = (e.n) la_j + W_m^T lg_j,  lf_j += (d f_bc / d f_j)^T c,  lbval += (d f_bc / d bval)^T c
__global__ void __launch_bounds__(kTile) k_adj_bndT(const double *__restrict__ fs, const double *__restrict__ la,
                                                    const double *__restrict__ lg, double *__restrict__ lf,
                                                    double *__restrict__ lbval, Geo<double> G,
                                                    const double *__restrict__ lbf) {
    const int j = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    int nbnd = 0;
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + j];
        nbnd += (nb < 0 && nb != kNone) ? 1 : 0;
    }
    if (nbnd == 0) return;
    const double rho0 = G.ip[G.tile_inst[blockIdx.x]].rho0;
    double lfj[kQ], fj[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lfj[a] = lf[a * np + j];
        fj[a] = fs[a * np + j];
    }
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + j];
        if (nb >= 0 || nb == kNone) continue;
        const int bf = -nb - 1;
        const double snx = G.sn[(2 * m) * np + j], sny = G.sn[(2 * m + 1) * np + j];
        const double wx = G.lsq[(2 * m) * np + j], wy = G.lsq[(2 * m + 1) * np + j];
        double c[kQ], bv3[3], lb3[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < kQ; ++a)
            c[a] = edot<double>(a, snx, sny) * la[a * np + j] + wx * lg[(2 * a) * np + j] +
                   wy * lg[(2 * a + 1) * np + j] + (lbf != nullptr ? lbf[(a * 4 + m) * np + j] : 0.0);
        adj_bv3(G, bf, bv3);
        adj_bvals_T(G.btype[bf], bv3, snx, sny, fj, rho0, c, lfj, lb3);
        if (lbval != nullptr)
            for (int q = 0; q < 3; ++q) lbval[q * G.nbt + bf] += lb3[q];
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
    const double dt = cell_dt(G, G.ip[G.tile_inst[blockIdx.x]], i);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        const double l = L[a * np + i];
        lf3[a * np + i] = l;
        lc[a * np + i] = l;
        la[a * np + i] = -(dt * (1.0 / 3.0)) * l;
    }
}

// ---- stage 2: from lf3, lc -> lB, la2.  Forward: X = B - dt/2 a2, f3 = (X + zt f^eq(X)) / (1 + zt)
// with zt = (dt/3)/tau (Eq. (fnewstage), J = 3), C' = C + dt/6 a2.
__global__ void __launch_bounds__(kTile) k_adj_stage2(const double *__restrict__ Bv, const double *__restrict__ f2,
                                                      const double *__restrict__ g2, const double *__restrict__ tau,
                                                      const double *__restrict__ lf3, const double *__restrict__ lc,
                                                      double *__restrict__ lB, double *__restrict__ la,
                                                      double *__restrict__ ltau, Geo<double> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    const double dt = cell_dt(G, P, i);
    double acc[kQ], X[kQ], mu[kQ], lX[kQ];
    adj_flux_acc(i, f2, g2, G, P.rho0, acc);
    const double zt = dt * (1.0 / 3.0) * (1.0 / tau[i]);
    const double inv = 1.0 / (1.0 + zt);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        X[a] = Bv[a * np + i] - 0.5 * dt * acc[a];
        const double l3 = lf3[a * np + i];
        lX[a] = inv * l3;
        mu[a] = zt * inv * l3;
    }
    if (ltau != nullptr) {  // d f3 / d zt = (f^eq(X) - X) / (1 + zt)^2, d zt / d tau = -zt / tau
        double eq[kQ], dr, r, u, v, l_z = 0.0;
        moments(X, P.rho0, dr, r, u, v);
        feq_dev(dr, r, u, v, eq);
#pragma unroll
        for (int a = 0; a < kQ; ++a) l_z += lf3[a * np + i] * (eq[a] - X[a]);
        ltau[i] = -l_z * inv * inv * zt / tau[i];
    }
    feq_vjp(X, P.rho0, mu, lX);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lB[a * np + i] = lX[a];
        la[a * np + i] = -0.5 * dt * lX[a] + dt * (1.0 / 6.0) * lc[a * np + i];
    }
}

// ---- stage 1: from lf2, lB, lc -> lf0 (=), la1.  Forward (z = dt/tau, zq = z/4, s = z/(1 + zq);
// s1 = s, or from tau1 under the per-stage SST reading):
//   X = f0 - dt/2 a1,  f2 = (X + zq f^eq(X)) / (1 + zq),
//   B = X + (s1/3) (f^eq(f0) - f0) + (s/3) (f^eq(X) - X),  C = dt/6 a1.
// ltau (and ltau1 when tau1 is given) receive the adjoints of the relaxation times (added).
__global__ void __launch_bounds__(kTile) k_adj_stage1(const double *__restrict__ f0, const double *__restrict__ s1,
                                                      const double *__restrict__ g1, const double *__restrict__ tau,
                                                      const double *__restrict__ lf2, const double *__restrict__ lB,
                                                      const double *__restrict__ lc, double *__restrict__ lf0,
                                                      double *__restrict__ la, double *__restrict__ ltau,
                                                      Geo<double> G, const double *__restrict__ tau1,
                                                      double *__restrict__ ltau1) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    const double dt = cell_dt(G, P, i);
    double acc[kQ], x0[kQ], X[kQ], lX[kQ], mu[kQ], lb[kQ];
    adj_flux_acc(i, s1, g1, G, P.rho0, acc);
    const double z = dt * (1.0 / tau[i]);
    const double zq = z * 0.25;
    const double inv = 1.0 / (1.0 + zq);
    const double s3 = z * inv * (1.0 / 3.0);  // the stage-2 collision term's share of B
    const double z1 = tau1 != nullptr ? dt / tau1[i] : z;
    const double inv1 = tau1 != nullptr ? 1.0 / (1.0 + 0.25 * z1) : inv;
    const double s31 = tau1 != nullptr ? z1 * inv1 * (1.0 / 3.0) : s3;  // the stage-1 term's
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        x0[a] = f0[a * np + i];
        X[a] = x0[a] - 0.5 * dt * acc[a];
        const double l2 = lf2[a * np + i];
        lb[a] = lB[a * np + i];
        lX[a] = inv * l2 + (1.0 - s3) * lb[a];
        mu[a] = zq * inv * l2 + s3 * lb[a];
    }
    if (ltau != nullptr) {
        // z = dt/tau: d f2 / d z = (f^eq(X) - X) inv^2 / 4; B carries (s/3)(f^eq(X) - X) and
        // (s1/3)(f^eq(f0) - f0) with s = z inv, ds/dz = inv^2 (s1 likewise in z1)
        double e1[kQ], e2[kQ], dr, r, u, v, l_z = 0.0, l_z1 = 0.0;
        moments(X, P.rho0, dr, r, u, v);
        feq_dev(dr, r, u, v, e2);
        moments(x0, P.rho0, dr, r, u, v);
        feq_dev(dr, r, u, v, e1);
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            l_z += lf2[a * np + i] * (e2[a] - X[a]) * 0.25 + lb[a] * (1.0 / 3.0) * (e2[a] - X[a]);
            l_z1 += lb[a] * (1.0 / 3.0) * (e1[a] - x0[a]);
        }
        const double lt = -l_z * inv * inv * z / tau[i];
        if (tau1 != nullptr) {
            ltau[i] += lt;
            ltau1[i] += -l_z1 * inv1 * inv1 * z1 / tau1[i];
        } else {
            ltau[i] += lt - l_z1 * inv * inv * z / tau[i];
        }
    }
    feq_vjp(X, P.rho0, mu, lX);
    double l0[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        l0[a] = lX[a] - s31 * lb[a];
        mu[a] = s31 * lb[a];
    }
    feq_vjp(x0, P.rho0, mu, l0);
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        lf0[a * np + i] = l0[a];
        la[a * np + i] = -0.5 * dt * lX[a] + dt * (1.0 / 6.0) * lc[a * np + i];
    }
}

// ---- relaxation of stage 1: lf0 += (d s1 / d f0)^T ls1, s1 = (f0 + zq f^eq(f0)) / (1 + zq)
__global__ void __launch_bounds__(kTile) k_adj_relax(const double *__restrict__ f0, const double *__restrict__ tau,
                                                     const double *__restrict__ ls1, double *__restrict__ lf0,
                                                     double *__restrict__ ltau, Geo<double> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    const double zq = cell_dt(G, P, i) / tau[i] * 0.25;
    const double inv = 1.0 / (1.0 + zq);
    double x0[kQ], l0[kQ], mu[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        x0[a] = f0[a * np + i];
        const double l1 = ls1[a * np + i];
        l0[a] = lf0[a * np + i] + inv * l1;
        mu[a] = zq * inv * l1;
    }
    if (ltau != nullptr) {  // d s1 / d zq = (f^eq(f0) - f0) / (1 + zq)^2, zq = dt / (4 tau)
        double eq[kQ], dr, r, u, v, l_z = 0.0;
        moments(x0, P.rho0, dr, r, u, v);
        feq_dev(dr, r, u, v, eq);
#pragma unroll
        for (int a = 0; a < kQ; ++a) l_z += ls1[a * np + i] * (eq[a] - x0[a]);
        ltau[i] += -l_z * inv * inv * zq / tau[i];
    }
    feq_vjp(x0, P.rho0, mu, l0);
#pragma unroll
    for (int a = 0; a < kQ; ++a) lf0[a * np + i] = l0[a];
}

// ---- explicit Euler comparison scheme: f^{n+1} = f + dt (-acc(f) + (f^eq(f) - f) / tau).
// From L (adjoint of f^{n+1}): lf0 = L + (dt/tau) (J_feq^T L - L) (=), la = -dt L, and the
// relaxation time's adjoint -dt/tau^2 sum L (f^eq - f) (=).
__global__ void __launch_bounds__(kTile) k_adj_euler(const double *__restrict__ f0, const double *__restrict__ tau,
                                                     const double *__restrict__ L, double *__restrict__ lf0,
                                                     double *__restrict__ la, double *__restrict__ ltau,
                                                     Geo<double> G) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    const double dt = cell_dt(G, P, i), c = dt / tau[i];
    double x0[kQ], l0[kQ], mu[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
        x0[a] = f0[a * np + i];
        const double l = L[a * np + i];
        l0[a] = (1.0 - c) * l;
        mu[a] = c * l;
        la[a * np + i] = -dt * l;
    }
    if (ltau != nullptr) {
        double eq[kQ], dr, r, u, v, s = 0.0;
        moments(x0, P.rho0, dr, r, u, v);
        feq_dev(dr, r, u, v, eq);
#pragma unroll
        for (int a = 0; a < kQ; ++a) s += L[a * np + i] * (eq[a] - x0[a]);
        ltau[i] = -s * c / tau[i];
    }
    feq_vjp(x0, P.rho0, mu, l0);
#pragma unroll
    for (int a = 0; a < kQ; ++a) lf0[a * np + i] = l0[a];
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

#include "fvlbm_adjoint_sst.cuh"

namespace {

// Device buffers of one adjoint call: one allocation, carved in 256-byte aligned pieces, freed
// when the call returns.  The carving runs twice: once to measure, once on the allocation.
struct AdjScratch {
    char *base = nullptr;
    size_t off = 0;
    ~AdjScratch() {
        if (base) cudaFree(base);
    }
    double *get(size_t n) {
        const size_t b = (std::max<size_t>(n, 2) * sizeof(double) + 255) / 256 * 256;
        double *p = base ? reinterpret_cast<double *>(base + off) : nullptr;
        off += b;
        return p;
    }
    cudaError_t allocate() {
        const size_t total = off;
        off = 0;
        return cudaMalloc(reinterpret_cast<void **>(&base), total);
    }
};

// The state a step starts from: f and, for SST handles, the macros (rho, u, v) of f, k, omega
// and nu_t (laminar handles: NULL).
struct AdjState {
    double *f = nullptr, *mac = nullptr, *k = nullptr, *w = nullptr, *nt = nullptr;
};

// Stage values of one step that its adjoint reads (SST: also the SST gradients [12 np], f1 and
// the step's tau; laminar: tau is the handle's).
struct AdjStep {
    double *s1, *g1, *f2, *g2, *B, *C, *f3, *g3, *mac;
    double *sg = nullptr, *f1 = nullptr, *tau = nullptr;
    // per-stage SST reading: the solves before stages 1 and 2 (their gradients, f1, tau) and the
    // macros of f^(1), f^(2) they read; the solve before stage 3 uses sg, f1, tau above
    double *sgA = nullptr, *f1A = nullptr, *tauA = nullptr, *sgB = nullptr, *f1B = nullptr, *tauB = nullptr;
    double *mac1 = nullptr, *mac2 = nullptr;
    double *kS = nullptr, *wS = nullptr, *ntS = nullptr;  // discarded k, omega, nu_t of those solves
};

// One two-pass FP64 step from state `in` to state `out` (the launches of the handle's two-pass
// path for its scheme and readings: the SST solve first on SST handles, three of them under the
// per-stage reading), with the stage values kept in S.
void adj_forward_step(fvlbm_handle *h, const Geo<double> &G, const AdjState &in, const AdjState &out,
                      const AdjStep &S) {
    const dim3 grid(h->ntiles), block(kTile);
    cudaStream_t s = h->stream;
    const double *tau = static_cast<const double *>(h->tau);
    double *mac_out = S.mac;
    auto solve = [&](const double *mac, double *sg, double *f1, double *ko, double *wo, double *nto,
                     double *tau_out) {
        const CompactGeo<double> CG{nullptr, nullptr};
        sst_grad_twopass<double>(h, mac, in.k, in.w, sg, f1, G, CG);
        sst_update_twopass<double>(h, mac, in.k, in.w, in.nt, sg, f1, ko, wo, nto, tau_out, G, CG);
    };
    if (h->scheme == 1) {  // explicit Euler: the SST solve, then one flux + collision update
        if (h->sst) solve(in.mac, S.sg, S.f1, out.k, out.w, out.nt, S.tau);
        grad_f<double>(h, grid, block, s, in.f, S.g1, G);
        k_flux_stage<double, 4, false><<<grid, block, 0, s>>>(in.f, S.g1, out.f, in.f, S.B, S.C,
                                                              h->sst ? S.tau : tau, h->sst ? out.mac : S.mac,
                                                              nullptr, G);
        return;
    }
    if (h->per_stage) {
        // the SST solved from t^n before every stage with the macros of f^n, f^(1), f^(2); stage 1
        // relaxes with the first tau, its algebra takes the second for f^(2); the last solve
        // gives the state of t^{n+1} and the tau of stages 2 and 3
        solve(in.mac, S.sgA, S.f1A, S.kS, S.wS, S.ntS, S.tauA);
        k_stage1<double><<<grid, block, 0, s>>>(in.f, S.s1, S.tauA, G);
        k_stage_macros<double><<<grid, block, 0, s>>>(S.s1, S.mac1, G);
        solve(S.mac1, S.sgB, S.f1B, S.kS, S.wS, S.ntS, S.tauB);
        grad_f<double>(h, grid, block, s, S.s1, S.g1, G);
        k_flux_stage<double, 1, false><<<grid, block, 0, s>>>(S.s1, S.g1, S.f2, in.f, S.B, S.C, S.tauB, S.mac,
                                                              nullptr, G, S.tauA);
        k_stage_macros<double><<<grid, block, 0, s>>>(S.f2, S.mac2, G);
        solve(S.mac2, S.sg, S.f1, out.k, out.w, out.nt, S.tau);
        grad_f<double>(h, grid, block, s, S.f2, S.g2, G);
        k_flux_stage<double, 2, false><<<grid, block, 0, s>>>(S.f2, S.g2, S.f3, in.f, S.B, S.C, S.tau, S.mac,
                                                              nullptr, G);
        grad_f<double>(h, grid, block, s, S.f3, S.g3, G);
        k_flux_stage<double, 3, false><<<grid, block, 0, s>>>(S.f3, S.g3, nullptr, out.f, S.B, S.C, S.tau,
                                                              out.mac, nullptr, G);
        return;
    }
    if (h->sst) {
        const CompactGeo<double> CG{nullptr, nullptr};
        sst_grad_twopass<double>(h, in.mac, in.k, in.w, S.sg, S.f1, G, CG);
        sst_update_twopass<double>(h, in.mac, in.k, in.w, in.nt, S.sg, S.f1, out.k, out.w, out.nt, S.tau, G, CG);
        tau = S.tau;
        mac_out = out.mac;
    }
    double *fin = in.f;
    k_stage1<double><<<grid, block, 0, s>>>(in.f, S.s1, tau, G);
    grad_f<double>(h, grid, block, s, S.s1, S.g1, G);
    k_flux_stage<double, 1, false><<<grid, block, 0, s>>>(S.s1, S.g1, S.f2, fin, S.B, S.C, tau, S.mac,
                                                          nullptr, G);
    grad_f<double>(h, grid, block, s, S.f2, S.g2, G);
    k_flux_stage<double, 2, false><<<grid, block, 0, s>>>(S.f2, S.g2, S.f3, fin, S.B, S.C, tau, S.mac,
                                                          nullptr, G);
    grad_f<double>(h, grid, block, s, S.f3, S.g3, G);
    k_flux_stage<double, 3, false><<<grid, block, 0, s>>>(S.f3, S.g3, nullptr, out.f, S.B, S.C, tau,
                                                          mac_out, nullptr, G);
}

// Adjoint variables.  L is the adjoint of f^{n+1} on entry to a step's reverse and of f^n on
// exit; lk, lw, lnt those of k, omega, nu_t (SST); lbval [5][nbt] accumulates the boundary
// values' adjoints.
struct AdjVars {
    double *L, *lf3, *lc, *la, *lg, *lB, *lf2, *ls1, *lf0, *lbval;
    double *a_sn = nullptr, *a_lsq = nullptr, *a_rown = nullptr, *a_rnbr = nullptr;  // shape adjoint
    double *a_bnrm = nullptr, *a_blen = nullptr;
    double *a_dinv = nullptr, *a_wd = nullptr;  // shape adjoint, SST only
    double *a_area = nullptr;                     // shape adjoint, limiter on grad f only
    double *lk = nullptr, *lw = nullptr, *lnt = nullptr, *ltau = nullptr;  // SST
    double *own = nullptr, *fbu = nullptr, *fbg = nullptr;
    // per-stage SST reading: the state adjoints of t^n as the three solves add them up, the
    // adjoints of the first two relaxation times, and zeros for the discarded solve outputs
    double *lkN = nullptr, *lwN = nullptr, *lntN = nullptr, *ltauA = nullptr, *ltauB = nullptr, *zero = nullptr;
    double *lnb = nullptr, *lbf = nullptr;  // limiter on grad f (reading variant 1)
};

// Reverse of the step that went from state `in` (stage values S): L <- adjoint of f^n, and on
// SST handles (lk, lw, lnt) <- adjoints of (k, omega, nu_t)^n.
void adj_backward_step(fvlbm_handle *h, const Geo<double> &G, const AdjState &in, const AdjStep &S,
                       AdjVars &A) {
    const dim3 grid(h->ntiles), block(kTile);
    cudaStream_t s = h->stream;
    const size_t nq = static_cast<size_t>(kQ) * h->np;
    const double *tau = h->sst ? S.tau : static_cast<const double *>(h->tau);
    const int *back = h->d_back;
    const double *f0 = in.f;
    auto geom = [&](const double *fs, const double *g) {
        if (A.a_sn)
            k_adj_geom<<<grid, block, 0, s>>>(fs, g, A.la, A.lg, G, A.a_sn, A.a_lsq, A.a_rown, A.a_rnbr);
    };
    // transpose of one flux + gradient evaluation at stage value fs (gradient g): la -> lf
    auto evalT = [&](const double *fs, const double *g, double *lf) {
        k_adj_fluxT<<<grid, block, 0, s>>>(A.la, lf, A.lg, G, back);
        if (A.lnb) k_adj_limT<<<grid, block, 0, s>>>(fs, A.lg, lf, A.lnb, A.lbf, G, A.a_rown, A.a_area);
        geom(fs, g);
        k_adj_gradT<<<grid, block, 0, s>>>(A.lg, lf, G, back, A.lnb);
        k_adj_bndT<<<grid, block, 0, s>>>(fs, A.la, A.lg, lf, A.lbval, G, A.lbf);
    };
    if (h->scheme == 1) {
        k_adj_euler<<<grid, block, 0, s>>>(f0, tau, A.L, A.lf0, A.la, A.ltau, G);
        evalT(f0, S.g1, A.lf0);
        if (h->sst) {
            const AdjGeo AG{A.a_sn, A.a_rown, A.a_rnbr, A.a_lsq, A.a_dinv, A.a_wd};
            k_adj_sst_update<<<grid, block, 0, s>>>(in.mac, in.k, in.w, in.nt, S.sg, S.f1, A.lk, A.lw, A.lnt,
                                                    A.ltau, A.own, A.fbu, A.lbval, G, AG);
            k_adj_sst_grad<<<grid, block, 0, s>>>(in.mac, in.k, in.w, S.sg, S.f1, A.fbu, A.own, A.fbg, A.lbval, G,
                                                  back, AG);
            k_adj_sst_finish<<<grid, block, 0, s>>>(f0, A.own, A.fbu, A.fbg, A.lf0, A.lk, A.lw, A.lnt, G, back,
                                                    false);
        }
        std::swap(A.L, A.lf0);
        return;
    }
    k_adj_stage3<<<grid, block, 0, s>>>(A.L, A.lf3, A.lc, A.la, G);
    evalT(S.f3, S.g3, A.lf3);
    k_adj_stage2<<<grid, block, 0, s>>>(S.B, S.f2, S.g2, tau, A.lf3, A.lc, A.lB, A.la, A.ltau, G);
    if (h->per_stage) {
        const size_t nb1 = static_cast<size_t>(h->np) * sizeof(double);
        const AdjGeo AG{A.a_sn, A.a_rown, A.a_rnbr, A.a_lsq, A.a_dinv, A.a_wd};
        // reverse of one SST solve from t^n with macros of fs: outputs' adjoints (lk, lw, lnt,
        // ltau) -> lf (through the macros) and the t^n state adjoints (lkN.. written or added)
        auto solveT = [&](const double *mac, const double *sg, const double *f1, const double *lk,
                          const double *lw, const double *lnt, const double *ltau, const double *fs, double *lf,
                          bool add) {
            k_adj_sst_update<<<grid, block, 0, s>>>(mac, in.k, in.w, in.nt, sg, f1, lk, lw, lnt, ltau, A.own, A.fbu,
                                                    A.lbval, G, AG);
            k_adj_sst_grad<<<grid, block, 0, s>>>(mac, in.k, in.w, sg, f1, A.fbu, A.own, A.fbg, A.lbval, G, back,
                                                  AG);
            k_adj_sst_finish<<<grid, block, 0, s>>>(fs, A.own, A.fbu, A.fbg, lf, A.lkN, A.lwN, A.lntN, G, back, add);
        };
        cudaMemsetAsync(A.lf2, 0, nq * sizeof(double), s);
        solveT(S.mac2, S.sg, S.f1, A.lk, A.lw, A.lnt, A.ltau, S.f2, A.lf2, false);
        evalT(S.f2, S.g2, A.lf2);
        cudaMemsetAsync(A.ltauA, 0, nb1, s);
        cudaMemsetAsync(A.ltauB, 0, nb1, s);
        k_adj_stage1<<<grid, block, 0, s>>>(f0, S.s1, S.g1, S.tauB, A.lf2, A.lB, A.lc, A.lf0, A.la, A.ltauB, G,
                                            S.tauA, A.ltauA);
        cudaMemsetAsync(A.ls1, 0, nq * sizeof(double), s);
        solveT(S.mac1, S.sgB, S.f1B, A.zero, A.zero, A.zero, A.ltauB, S.s1, A.ls1, true);
        evalT(S.s1, S.g1, A.ls1);
        k_adj_relax<<<grid, block, 0, s>>>(f0, S.tauA, A.ls1, A.lf0, A.ltauA, G);
        solveT(in.mac, S.sgA, S.f1A, A.zero, A.zero, A.zero, A.ltauA, f0, A.lf0, true);
        std::swap(A.L, A.lf0);
        std::swap(A.lk, A.lkN);
        std::swap(A.lw, A.lwN);
        std::swap(A.lnt, A.lntN);
        return;
    }
    cudaMemsetAsync(A.lf2, 0, nq * sizeof(double), s);
    evalT(S.f2, S.g2, A.lf2);
    k_adj_stage1<<<grid, block, 0, s>>>(f0, S.s1, S.g1, tau, A.lf2, A.lB, A.lc, A.lf0, A.la, A.ltau, G, nullptr,
                                        nullptr);
    cudaMemsetAsync(A.ls1, 0, nq * sizeof(double), s);
    evalT(S.s1, S.g1, A.ls1);
    k_adj_relax<<<grid, block, 0, s>>>(f0, tau, A.ls1, A.lf0, A.ltau, G);
    if (h->sst) {
        const AdjGeo AG{A.a_sn, A.a_rown, A.a_rnbr, A.a_lsq, A.a_dinv, A.a_wd};
        k_adj_sst_update<<<grid, block, 0, s>>>(in.mac, in.k, in.w, in.nt, S.sg, S.f1, A.lk, A.lw, A.lnt, A.ltau,
                                                A.own, A.fbu, A.lbval, G, AG);
        k_adj_sst_grad<<<grid, block, 0, s>>>(in.mac, in.k, in.w, S.sg, S.f1, A.fbu, A.own, A.fbg, A.lbval, G,
                                              back, AG);
        k_adj_sst_finish<<<grid, block, 0, s>>>(f0, A.own, A.fbu, A.fbg, A.lf0, A.lk, A.lw, A.lnt, G, back, false);
    }
    std::swap(A.L, A.lf0);
}

int adjoint_impl(fvlbm_handle *h, int instance, int n_steps, const double *w, double *J, double *dJ_df,
                 double *dJ_dbedge, double *dJ_dxy, double *cdcl = nullptr) {
    if (!h || instance < 0 || instance >= h->ninst || n_steps < 0 || !w) return FVLBM_ERR_BAD_PARAM;
    if (h->precision != FVLBM_FP64 || h->d_back == nullptr)
        return FVLBM_ERR_NOT_SUPPORTED;
    const InstInfo &I = h->inst[instance];
    if (dJ_dxy && (!I.mesh || !I.mesh->ppairs.empty())) return FVLBM_ERR_NOT_SUPPORTED;
    CK(cudaSetDevice(h->device));
    const Geo<double> G = geo_of<double>(h);
    const bool sst = h->sst;
    const size_t np = h->np, nq = static_cast<size_t>(kQ) * np;
    // Memory plan.  The stage values one adjoint step reads take 99 doubles per cell (f^n, f^(1),
    // f^(2), B, f^(3) and the three gradients; SST adds 20: the macros, k, omega, nu_t, the SST
    // gradients, f1 and tau; the per-stage reading 34 more for its two extra solves and the
    // macros they read); a state snapshot takes 9 (SST: 15).  Within the budget (the
    // handle's adjoint budget, else half the free device memory) all steps keep their stage
    // values when they fit, and every step runs forward once.  Otherwise the run is cut into
    // units of K steps whose stage values fit in half the budget, the other half holds c state
    // snapshots, and the units are reversed on a binomial (revolve) schedule: with c snapshots
    // and r forward passes per unit at most, C(c + r, c) units can be reversed, and r is the
    // least such number.  With a snapshot for every unit start that is r = 1: each unit runs
    // forward twice (once to reach the next snapshot, once keeping its stage values).
    const bool ps = h->per_stage;
    const size_t per_step = (ps ? 153 : (sst ? 119 : 99)) * np * sizeof(double);
    const size_t per_snap = (sst ? 15 : 9) * np * sizeof(double);
    size_t budget = h->adj_budget;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        budget = fr / 2;
    }
    int K = std::max(n_steps, 1), nsnap = 0;
    if (static_cast<size_t>(n_steps) * per_step > budget) {
        K = static_cast<int>(std::max<size_t>(1, budget / 2 / per_step));
        const int units = (n_steps + K - 1) / K;
        const size_t left = budget > K * per_step ? budget - K * per_step : 0;
        nsnap = static_cast<int>(std::min<size_t>(units - 1, std::max<size_t>(1, left / per_snap)));
    }
    const int units = n_steps > 0 ? (n_steps + K - 1) / K : 0;
    AdjScratch M;
    double *Cs, *macs, *kS = nullptr, *wS = nullptr, *ntS = nullptr;
    AdjState xa, xb;
    std::vector<AdjState> snap(nsnap), st(K);
    std::vector<AdjStep> slot(K);
    AdjVars A{};
    const size_t nbt = std::max(h->nbt, 1);
    auto state = [&](AdjState &x) {
        x.f = M.get(nq);
        if (sst) {
            x.mac = M.get(3 * np);
            x.k = M.get(np);
            x.w = M.get(np);
            x.nt = M.get(np);
        }
    };
    auto carve = [&] {
        state(xa);
        state(xb);
        Cs = M.get(nq);
        macs = M.get(3 * np);
        if (ps) {
            kS = M.get(np);
            wS = M.get(np);
            ntS = M.get(np);
        }
        for (auto &x : snap) state(x);
        for (int k = 0; k < K; ++k) {
            state(st[k]);
            slot[k].s1 = M.get(nq);
            slot[k].g1 = M.get(2 * nq);
            slot[k].f2 = M.get(nq);
            slot[k].g2 = M.get(2 * nq);
            slot[k].B = M.get(nq);
            slot[k].C = Cs;
            slot[k].f3 = M.get(nq);
            slot[k].g3 = M.get(2 * nq);
            slot[k].mac = macs;
            if (sst) {
                slot[k].sg = M.get(12 * np);
                slot[k].f1 = M.get(np);
                slot[k].tau = M.get(np);
            }
            if (ps) {
                slot[k].sgA = M.get(12 * np);
                slot[k].f1A = M.get(np);
                slot[k].tauA = M.get(np);
                slot[k].sgB = M.get(12 * np);
                slot[k].f1B = M.get(np);
                slot[k].tauB = M.get(np);
                slot[k].mac1 = M.get(3 * np);
                slot[k].mac2 = M.get(3 * np);
                slot[k].kS = kS;
                slot[k].wS = wS;
                slot[k].ntS = ntS;
            }
        }
        A.L = M.get(nq);
        A.lf3 = M.get(nq);
        A.lc = M.get(nq);
        A.la = M.get(nq);
        A.lg = M.get(2 * nq);
        A.lB = M.get(nq);
        A.lf2 = M.get(nq);
        A.ls1 = M.get(nq);
        A.lf0 = M.get(nq);
        A.lbval = M.get(5 * nbt);
        if (sst) {
            A.lk = M.get(np);
            A.lw = M.get(np);
            A.lnt = M.get(np);
            A.ltau = M.get(np);
            A.own = M.get(kSstOwn * np);
            A.fbu = M.get(4 * kSstFU * np);
            A.fbg = M.get(4 * kSstFG * np);
        }
        if (ps) {
            A.lkN = M.get(np);
            A.lwN = M.get(np);
            A.lntN = M.get(np);
            A.ltauA = M.get(np);
            A.ltauB = M.get(np);
            A.zero = M.get(np);
        }
        if (h->limit_f) {
            A.lnb = M.get(4 * kQ * np);
            A.lbf = M.get(4 * kQ * np);
        }
        if (dJ_dxy) {
            A.a_sn = M.get(8 * np);
            A.a_lsq = M.get(8 * np);
            A.a_rown = M.get(8 * np);
            A.a_rnbr = M.get(8 * np);
            A.a_bnrm = M.get(2 * nbt);
            A.a_blen = M.get(nbt);
            if (sst) {
                A.a_dinv = M.get(4 * np);
                A.a_wd = M.get(np);
            }
            if (h->limit_f) A.a_area = M.get(np);
        }
    };
    carve();
    CK(M.allocate());
    carve();
    cudaStream_t s = h->stream;
    if (dJ_dxy) {
        for (double *x : {A.a_sn, A.a_lsq, A.a_rown, A.a_rnbr})
            CK(cudaMemsetAsync(x, 0, 8 * np * sizeof(double), s));
        CK(cudaMemsetAsync(A.a_bnrm, 0, 2 * nbt * sizeof(double), s));
        CK(cudaMemsetAsync(A.a_blen, 0, nbt * sizeof(double), s));
        if (sst) {
            CK(cudaMemsetAsync(A.a_dinv, 0, 4 * np * sizeof(double), s));
            CK(cudaMemsetAsync(A.a_wd, 0, np * sizeof(double), s));
        }
        if (A.a_area) CK(cudaMemsetAsync(A.a_area, 0, np * sizeof(double), s));
    }
    if (sst) {  // J does not depend on k, omega, nu_t of the last state
        for (double *x : {A.lk, A.lw, A.lnt}) CK(cudaMemsetAsync(x, 0, np * sizeof(double), s));
        // laminar instances of the batch keep the handle's tau (the SST kernels skip them)
        for (int k = 0; k < K; ++k)
            for (double *t : {slot[k].tau, slot[k].tauA, slot[k].tauB})
                if (t) CK(cudaMemcpyAsync(t, h->tau, np * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (ps) CK(cudaMemsetAsync(A.zero, 0, np * sizeof(double), s));
    }
    auto copy_state = [&](const AdjState &dst, const AdjState &src) -> int {
        CK(cudaMemcpyAsync(dst.f, src.f, nq * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (sst) {
            CK(cudaMemcpyAsync(dst.mac, src.mac, 3 * np * sizeof(double), cudaMemcpyDeviceToDevice, s));
            for (int q = 0; q < 3; ++q) {
                double *d = q == 0 ? dst.k : (q == 1 ? dst.w : dst.nt);
                const double *c = q == 0 ? src.k : (q == 1 ? src.w : src.nt);
                CK(cudaMemcpyAsync(d, c, np * sizeof(double), cudaMemcpyDeviceToDevice, s));
            }
        }
        return FVLBM_OK;
    };
    AdjState h0;  // the handle's current state
    h0.f = static_cast<double *>(h->fn);
    if (sst) {
        h0.mac = static_cast<double *>(h->mac);
        h0.k = static_cast<double *>(h->kk[h->turb]);
        h0.w = static_cast<double *>(h->ww[h->turb]);
        h0.nt = static_cast<double *>(h->nut[h->turb]);
    }
    // steps k0 .. k1-1 from `start` with their stage values kept; the state after them into xb
    auto fill = [&](int k0, int k1, const AdjState &start) -> int {
        int rc = copy_state(st[0], start);
        if (rc) return rc;
        for (int n = k0; n < k1; ++n)
            adj_forward_step(h, G, st[n - k0], n + 1 < k1 ? st[n + 1 - k0] : xb, slot[n - k0]);
        CK(cudaGetLastError());
        return FVLBM_OK;
    };
    // units u0 .. u1-1 forward from `start` without keeping stage values; the state into `dst`
    auto advance = [&](int u0, int u1, const AdjState &start, const AdjState &dst) -> int {
        const int k0 = u0 * K, k1 = std::min(n_steps, u1 * K);
        if (k1 <= k0) return copy_state(dst, start);
        int rc = copy_state(xa, start);
        if (rc) return rc;
        for (int n = k0; n < k1; ++n) {
            adj_forward_step(h, G, xa, n + 1 < k1 ? xb : dst, slot[0]);
            std::swap(xa, xb);
        }
        CK(cudaGetLastError());
        return FVLBM_OK;
    };
    // J at f^N and its derivatives with respect to f^N: taken when the last unit has been filled
    // (its end state is f^N), before the first reverse step
    bool seeded = false;
    auto seed = [&](const double *fN) -> int {
        double out[4];
        int rc = forces_impl(h, instance, 0.0, out, nullptr, nullptr, fN);
        if (rc) return rc;
        if (J) *J = w[0] * out[2] + w[1] * out[3];
        if (cdcl) {
            cdcl[0] = out[2];
            cdcl[1] = out[3];
        }
        const double q = 0.5 * I.rho0 * I.uref * I.uref * I.lref;
        const double al = I.alpha_deg * M_PI / 180.0, ca = std::cos(al), sa = std::sin(al);
        const double cx = (w[0] * ca - w[1] * sa) / q, cy = (w[0] * sa + w[1] * ca) / q;
        CK(cudaMemsetAsync(A.lbval, 0, 5 * nbt * sizeof(double), s));
        k_adj_seed<<<h->ntiles, kTile, 0, s>>>(fN, static_cast<const double *>(h->bnrm),
                                               static_cast<const double *>(h->blen), instance, cx, cy, A.L,
                                               A.lbval, A.a_bnrm, A.a_blen, G);
        CK(cudaGetLastError());
        seeded = true;
        return FVLBM_OK;
    };
    // reverse one unit whose start state is `start`
    auto reverse_unit = [&](int u, const AdjState &start) -> int {
        const int k0 = u * K, k1 = std::min(n_steps, k0 + K);
        int rc = fill(k0, k1, start);
        if (rc) return rc;
        if (!seeded && (rc = seed(xb.f))) return rc;
        for (int n = k1 - 1; n >= k0; --n) adj_backward_step(h, G, st[n - k0], slot[n - k0], A);
        CK(cudaGetLastError());
        return FVLBM_OK;
    };
    if (n_steps == 0) {
        int rc = seed(h0.f);
        if (rc) return rc;
    } else {  // the units on the binomial schedule (host logic, revolve_schedule)
        std::vector<RevolveAction> plan;
        if (!revolve_schedule(units, nsnap, &plan)) return FVLBM_ERR_BAD_PARAM;
        for (const RevolveAction &act : plan) {
            const AdjState &from = act.from < 0 ? h0 : snap[act.from];
            int rc = act.kind == RevolveAction::kAdvance ? advance(act.u0, act.u1, from, snap[act.to])
                                                         : reverse_unit(act.u0, from);
            if (rc) return rc;
        }
    }
    double *xscr = xb.f;
    if (dJ_df && I.nc > 0) {
        k_adj_gather<<<(I.nc + 255) / 256, 256, 0, s>>>(A.L, h->d_perm + perm_offset(h, instance), I.cell_off,
                                                         I.nc, np, xscr);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(dJ_df, xscr, sizeof(double) * kQ * static_cast<size_t>(I.nc), cudaMemcpyDeviceToHost,
                           s));
    }
    std::vector<double> lb(5 * static_cast<size_t>(std::max(I.nb, 1)));
    if (dJ_dbedge && I.nb > 0)
        for (int c = 0; c < 5; ++c)
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
        runs.resize(4 * 8 * nc + 6 * nc + 3 * static_cast<size_t>(std::max(I.nb, 1)));
        const double *src[4] = {A.a_sn, A.a_lsq, A.a_rown, A.a_rnbr};
        for (int q = 0; q < 4; ++q)
            for (int c = 0; c < 8; ++c)
                CK(cudaMemcpyAsync(runs.data() + (8 * q + c) * nc, src[q] + c * np + I.cell_off, sizeof(double) * nc,
                                   cudaMemcpyDeviceToHost, s));
        if (sst) {  // 1 / |d| [4 runs] and the wall distance
            for (int c = 0; c < 4; ++c)
                CK(cudaMemcpyAsync(runs.data() + (32 + c) * nc, A.a_dinv + c * np + I.cell_off, sizeof(double) * nc,
                                   cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(runs.data() + 36 * nc, A.a_wd + I.cell_off, sizeof(double) * nc,
                               cudaMemcpyDeviceToHost, s));
        }
        if (A.a_area)  // the limiter's cell areas
            CK(cudaMemcpyAsync(runs.data() + 37 * nc, A.a_area + I.cell_off, sizeof(double) * nc,
                               cudaMemcpyDeviceToHost, s));
        double *bt = runs.data() + 38 * nc;
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
        if (sst) {
            GA.dinv.assign(4 * nc, 0.0);
            GA.wdist.assign(nc, 0.0);
            for (size_t k = 0; k < nc; ++k) {
                for (int l = 0; l < 4; ++l) GA.dinv[4 * static_cast<size_t>(perm[k]) + l] = runs[(32 + l) * nc + k];
                GA.wdist[perm[k]] = runs[36 * nc + k];
            }
        }
        if (A.a_area) {
            GA.area.assign(nc, 0.0);
            for (size_t k = 0; k < nc; ++k) GA.area[perm[k]] = runs[37 * nc + k];
        }
        const size_t nbe = mc.btype.size();
        GA.bnrm.assign(2 * nbe, 0.0);
        GA.blen.assign(nbe, 0.0);
        const double *bt = runs.data() + 38 * nc;
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
            for (int c = 0; c < 5; ++c)
                dJ_dbedge[5 * static_cast<size_t>(I.bedge_of[b]) + c] = lb[static_cast<size_t>(c) * I.nb + b];
    }
    return FVLBM_OK;
}

}  // namespace
