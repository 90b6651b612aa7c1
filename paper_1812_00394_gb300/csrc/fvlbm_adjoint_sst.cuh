// fvlbm_adjoint_sst.cuh -- reverse mode of the k-omega SST solve (Sec. 2; Sec. 3.2, Step 1) for
// the discrete adjoint; included by fvlbm_adjoint.cuh.
//
// Forward, per step (two-pass FP64 kernels, default reading): k_sst_grad forms the gradients of
// u, v, k, omega, the limited k / omega gradients and the blending f1 of every cell from its face
// neighbours (or boundary values); k_sst_update forms k', omega', nu_t' and tau = (nu + nu_t')/c_s^2
// from the cell, its neighbours' values, limited gradients, f1 and nu_t.  The adjoint inverts the
// order: the update, then the gradients, each transposed per cell in closed form.  A cell's
// adjoint with respect to a neighbour's value is written to a per-face buffer at the cell's own
// face slot; the neighbour gathers it through the face's back slot (no atomics, deterministic).
// Where the forward takes min / max / clip branches, the adjoint follows the branch the values
// took, with the tie-breaking of the tangent's fmin / fmax (ties keep the first argument).

namespace fvlbm {

// Adjoint of sst_bvals for boundary face b: la4 = adjoint of (u_b, v_b, k_b, omega_b) to the
// owner's (u, v, k, omega) (outlet) or to the boundary values (wall: u_b, v_b; inlet and far
// field: u_b, v_b, k_b, omega_b); lbval is [5][nbt] (NULL: boundary adjoints not kept).
__device__ __forceinline__ void sst_bvals_T(const Geo<double> &G, int b, const double *la4, double *lown,
                                            double *lbval) {
    const int t = G.btype[b];
    if (t == FVLBM_BC_OUTLET) {
#pragma unroll
        for (int c = 0; c < 4; ++c) lown[c] += la4[c];
    } else if (lbval != nullptr) {
        lbval[1 * G.nbt + b] += la4[0];
        lbval[2 * G.nbt + b] += la4[1];
        if (t != FVLBM_BC_WALL) {  // wall: k_b = 0, omega_b = 60 nu / (beta1 d^2) are fixed
            lbval[3 * G.nbt + b] += la4[2];
            lbval[4 * G.nbt + b] += la4[3];
        }
    }
}

// Adjoints of the geometry arrays the SST kernels read (all NULL: no shape gradient): n dl / A,
// face offsets r_own and r_nbr, least-squares weights, 1 / |d| and the wall distance.
struct AdjGeo {
    double *sn, *rown, *rnbr, *lsq, *dinv, *wd;
};

// Reverse of the non-orthogonal correction of face m: l_dkn, l_dwn (adjoints of the face's
// normal derivatives) to the own gradients l_g, the neighbour's gradients (lf[10..13]) and the
// face geometry.
__device__ __forceinline__ void sst_face_correction_T(const SstFace<double> &f, const double *g, double dla,
                                                      double l_dkn, double l_dwn, double *l_g, double *lf,
                                                      const AdjGeo &AG, int m, size_t np, int i) {
    double ax, ay, l_tx, l_ty;
    if (!f.bnd) {
        ax = f.rox - f.rnx;
        ay = f.roy - f.rny;
        const double tx = f.snx / dla - ax * f.dinv, ty = f.sny / dla - ay * f.dinv;
        l_g[4] += 0.5 * l_dkn * tx;
        l_g[5] += 0.5 * l_dkn * ty;
        l_g[6] += 0.5 * l_dwn * tx;
        l_g[7] += 0.5 * l_dwn * ty;
        lf[10] += 0.5 * l_dkn * tx;
        lf[11] += 0.5 * l_dkn * ty;
        lf[12] += 0.5 * l_dwn * tx;
        lf[13] += 0.5 * l_dwn * ty;
        l_tx = 0.5 * (l_dkn * (g[4] + f.gn[0]) + l_dwn * (g[6] + f.gn[2]));
        l_ty = 0.5 * (l_dkn * (g[5] + f.gn[1]) + l_dwn * (g[7] + f.gn[3]));
    } else {
        ax = f.rox;
        ay = f.roy;
        const double tx = f.snx / dla - ax * f.dinv, ty = f.sny / dla - ay * f.dinv;
        l_g[4] += l_dkn * tx;
        l_g[5] += l_dkn * ty;
        l_g[6] += l_dwn * tx;
        l_g[7] += l_dwn * ty;
        l_tx = l_dkn * g[4] + l_dwn * g[6];
        l_ty = l_dkn * g[5] + l_dwn * g[7];
    }
    if (AG.sn != nullptr) {  // t = n dl/A / |n dl/A| - a / |d|
        const double d3 = dla * dla * dla;
        AG.sn[(2 * m) * np + i] += l_tx * (1.0 / dla - f.snx * f.snx / d3) - l_ty * f.snx * f.sny / d3;
        AG.sn[(2 * m + 1) * np + i] += -l_tx * f.snx * f.sny / d3 + l_ty * (1.0 / dla - f.sny * f.sny / d3);
        AG.rown[(2 * m) * np + i] -= l_tx * f.dinv;
        AG.rown[(2 * m + 1) * np + i] -= l_ty * f.dinv;
        if (!f.bnd) {
            AG.rnbr[(2 * m) * np + i] += l_tx * f.dinv;
            AG.rnbr[(2 * m + 1) * np + i] += l_ty * f.dinv;
        }
        AG.dinv[m * np + i] -= l_tx * ax + l_ty * ay;
    }
}

// Per-face buffer layout: value c of face slot m of cell i at buf[(c * 4 + m) * np + i].
// Update buffer (14 values): adjoints of the neighbour's u, v, k, omega, limited gradients (4),
// f1, nu_t and (non-orthogonal correction, reading variant 2) its k / omega gradients (4).
// Gradient buffer (4 values): adjoints of the neighbour's u, v, k, omega.
constexpr int kSstFU = 14, kSstFG = 4;

// Normal derivatives of k and omega on one face as sst_cell_update forms them: the two-point
// difference and, under reading variant 2, the non-orthogonal correction with the mean (interior)
// or own (boundary) gradient along n - d/|d|.
__device__ __forceinline__ void sst_face_normal_gradients(const SstFace<double> &f, const double *g, double ki,
                                                          double wi, double dla, bool nonorth, double &dkn,
                                                          double &dwn) {
    dkn = (f.k - ki) * f.dinv;
    dwn = (f.w - wi) * f.dinv;
    if (!nonorth) return;
    if (!f.bnd) {
        const double tx = f.snx / dla - (f.rox - f.rnx) * f.dinv;
        const double ty = f.sny / dla - (f.roy - f.rny) * f.dinv;
        dkn += 0.5 * ((g[4] + f.gn[0]) * tx + (g[5] + f.gn[1]) * ty);
        dwn += 0.5 * ((g[6] + f.gn[2]) * tx + (g[7] + f.gn[3]) * ty);
    } else {
        const double tx = f.snx / dla - f.rox * f.dinv, ty = f.sny / dla - f.roy * f.dinv;
        dkn += g[4] * tx + g[5] * ty;
        dwn += g[6] * tx + g[7] * ty;
    }
}


// Own adjoints after the update: u, v, k, omega, nu_t, g[8], lg[4], f1 (18 values, [18][np]).
constexpr int kSstOwn = 18;

// ---- reverse of sst_cell_update (+ tau) of one cell.  In: lam_k', lam_w', lam_nt' (the latter
// including c_s^-2 lam_tau).  Out: own adjoints and the per-face neighbour adjoints.
__global__ void __launch_bounds__(kTile) k_adj_sst_update(
    const double *__restrict__ mac, const double *__restrict__ kk, const double *__restrict__ ww,
    const double *__restrict__ nut, const double *__restrict__ grads, const double *__restrict__ f1a,
    const double *__restrict__ lk1, const double *__restrict__ lw1, const double *__restrict__ lnt1,
    const double *__restrict__ ltau, double *__restrict__ own, double *__restrict__ fbuf,
    double *__restrict__ lbval, Geo<double> G, AdjGeo AG) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    if (!P.sst) return;
    const double nu = P.nu, dt = cell_dt(G, P, i);
    const double ui = mac[np + i], vi = mac[2 * np + i], ki = kk[i], wi = ww[i], nti = nut[i];
    const double di = G.wdist[i], f1 = f1a[i];
    const bool nonorth = (P.variant & 2) != 0;
    double g[8], lgi[4];
#pragma unroll
    for (int c = 0; c < 8; ++c) g[c] = grads[c * np + i];
#pragma unroll
    for (int c = 0; c < 4; ++c) lgi[c] = grads[(8 + c) * np + i];
    // ---------------- forward, keeping what the reverse needs
    const double sk_i = f1 * kSk1 + (1.0 - f1) * kSk2;
    const double sw_i = f1 * kSw1 + (1.0 - f1) * kSw2;
    double ck = 0, cw = 0, dk = 0, dw = 0;
    SstFace<double> F[4];
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + i];
        SstFace<double> &f = F[m];
        f.has = nb != kNone;
        if (!f.has) continue;
        f.bnd = nb < 0;
        f.snx = G.sn[(2 * m) * np + i];
        f.sny = G.sn[(2 * m + 1) * np + i];
        f.rox = G.rown[(2 * m) * np + i];
        f.roy = G.rown[(2 * m + 1) * np + i];
        f.dinv = G.dinv[m * np + i];
        if (nb >= 0) {
            f.u = mac[np + nb];
            f.v = mac[2 * np + nb];
            f.k = kk[nb];
            f.w = ww[nb];
            f.rnx = G.rnbr[(2 * m) * np + i];
            f.rny = G.rnbr[(2 * m + 1) * np + i];
#pragma unroll
            for (int c = 0; c < 4; ++c) f.lg[c] = grads[(8 + c) * np + nb];
#pragma unroll
            for (int c = 0; c < 4; ++c) f.gn[c] = grads[(4 + c) * np + nb];
            f.f1 = f1a[nb];
            f.nut = nut[nb];
        } else {
            sst_bvals(G, -nb - 1, nu, ui, vi, ki, wi, di, f.u, f.v, f.k, f.w);
        }
        const double kin = ki + lgi[0] * f.rox + lgi[1] * f.roy;
        const double win = wi + lgi[2] * f.rox + lgi[3] * f.roy;
        const double dla = sqrt(f.snx * f.snx + f.sny * f.sny);
        double dkn, dwn;
        sst_face_normal_gradients(f, g, ki, wi, dla, nonorth, dkn, dwn);
        if (!f.bnd) {
            const double un = 0.5 * (ui + f.u) * f.snx + 0.5 * (vi + f.v) * f.sny;
            const double kup = un >= 0.0 ? kin : f.k + f.lg[0] * f.rnx + f.lg[1] * f.rny;
            const double wup = un >= 0.0 ? win : f.w + f.lg[2] * f.rnx + f.lg[3] * f.rny;
            const double skj = f.f1 * kSk1 + (1.0 - f.f1) * kSk2;
            const double swj = f.f1 * kSw1 + (1.0 - f.f1) * kSw2;
            ck += un * kup;
            cw += un * wup;
            dk += 0.5 * ((nu + sk_i * nti) + (nu + skj * f.nut)) * dkn * dla;
            dw += 0.5 * ((nu + sw_i * nti) + (nu + swj * f.nut)) * dwn * dla;
        } else {
            const double un = f.u * f.snx + f.v * f.sny;
            ck += un * (un >= 0.0 ? kin : f.k);
            cw += un * (un >= 0.0 ? win : f.w);
            dk += (nu + sk_i * nti) * dkn * dla;
            dw += (nu + sw_i * nti) * dwn * dla;
        }
    }
    const double s11 = g[0], s22 = g[3], s12 = 0.5 * (g[1] + g[2]);
    const double SS = s11 * s11 + s22 * s22 + 2.0 * s12 * s12;
    const double dv = s11 + s22;
    const double Sabs = sqrt(2.0 * SS);
    const double cw1 = kB1 / kBstar - kSw1 * kKappa * kKappa / 0.3;
    const double cw2 = kB2 / kBstar - kSw2 * kKappa * kKappa / 0.3;
    const double gam = f1 * cw1 + (1.0 - f1) * cw2;
    const double Q = 2.0 * SS - (2.0 / 3.0) * dv * dv;
    const double pk0 = nti * Q - (2.0 / 3.0) * ki * dv;
    const double cap = 10.0 * kBstar * wi * ki;  // production limiter (reading variant 8)
    const bool capped = (P.variant & 8) && pk0 > cap;
    const double pk = capped ? cap : pk0;
    double pw = gam * Q;
    if (nti > 0.0) pw -= (2.0 / 3.0) * gam * ki * dv / nti;
    const double G46 = g[4] * g[6] + g[5] * g[7];
    const double cross = 2.0 * (1.0 - f1) * kSw2 / wi * G46;
    const double rk = -ck + dk + pk;
    const double rw = -cw + dw + pw + cross;
    const double beta = f1 * kB1 + (1.0 - f1) * kB2;
    const double Dk = 1.0 + dt * kBstar * wi, Dw = 1.0 + dt * beta * wi;
    const double kn0 = (ki + dt * rk) / Dk, wn0 = (wi + dt * rw) / Dw;
    const double kn = kn0 > 0.0 ? kn0 : 0.0;
    const double wn = wn0 > P.omega_min ? wn0 : P.omega_min;
    const double X1 = 2.0 * sqrt(kn) / (kBstar * wn * di), X2 = 500.0 * nu / (wn * di * di);
    const double arg2 = X2 > X1 ? X2 : X1;
    const double f2 = tanh(arg2 * arg2);
    const double A1 = kA1 * wn, B1 = Sabs * f2;
    const double Dn = B1 > A1 ? B1 : A1;
    const double ntn = kA1 * kn / Dn;
    // ---------------- reverse
    double l_kn = lk1[i], l_wn = lw1[i];
    const double l_nt = lnt1[i] + (ltau != nullptr ? ltau[i] / kCs2 : 0.0);
    double l_Sabs = 0, l_f1 = 0, l_ki = 0, l_wi = 0, l_nti = 0, l_ui = 0, l_vi = 0;
    double l_g[8] = {0, 0, 0, 0, 0, 0, 0, 0}, l_lgi[4] = {0, 0, 0, 0};
    l_kn += l_nt * kA1 / Dn;
    const double l_Dn = -l_nt * ntn / Dn;
    double l_f2 = 0.0;
    if (B1 > A1) {
        l_Sabs += l_Dn * f2;
        l_f2 = l_Dn * Sabs;
    } else {
        l_wn += l_Dn * kA1;
    }
    const double l_arg2 = l_f2 * (1.0 - f2 * f2) * 2.0 * arg2;
    double l_di = 0.0;
    if (X2 > X1) {
        l_wn -= l_arg2 * X2 / wn;
        l_di -= l_arg2 * 2.0 * X2 / di;
    } else {
        if (kn > 0.0) l_kn += l_arg2 / (kBstar * wn * di * sqrt(kn));
        l_wn -= l_arg2 * X1 / wn;
        l_di -= l_arg2 * X1 / di;
    }
    const double l_kn0 = kn0 > 0.0 ? l_kn : 0.0;
    const double l_wn0 = wn0 > P.omega_min ? l_wn : 0.0;
    l_ki += l_kn0 / Dk;
    const double l_rk = l_kn0 * dt / Dk;
    l_wi -= l_kn0 * kn0 * dt * kBstar / Dk;
    l_wi += l_wn0 / Dw;
    const double l_rw = l_wn0 * dt / Dw;
    const double l_Dw = -l_wn0 * wn0 / Dw;
    l_f1 += l_Dw * dt * wi * (kB1 - kB2);
    l_wi += l_Dw * dt * beta;
    const double l_ck = -l_rk, l_dk = l_rk, l_pk = l_rk;
    const double l_cw = -l_rw, l_dw = l_rw, l_pw = l_rw, l_cross = l_rw;
    // cross
    l_f1 -= l_cross * 2.0 * kSw2 / wi * G46;
    l_wi -= l_cross * cross / wi;
    {
        const double l_G = l_cross * 2.0 * (1.0 - f1) * kSw2 / wi;
        l_g[4] += l_G * g[6];
        l_g[6] += l_G * g[4];
        l_g[5] += l_G * g[7];
        l_g[7] += l_G * g[5];
    }
    // pw, pk
    double l_gam = l_pw * Q, l_Q = l_pw * gam, l_dv = 0.0;
    if (nti > 0.0) {
        const double t = (2.0 / 3.0) * gam * ki * dv / nti;
        l_gam -= l_pw * (2.0 / 3.0) * ki * dv / nti;
        l_ki -= l_pw * (2.0 / 3.0) * gam * dv / nti;
        l_dv -= l_pw * (2.0 / 3.0) * gam * ki / nti;
        l_nti += l_pw * t / nti;
    }
    const double l_pk0 = capped ? 0.0 : l_pk;
    if (capped) {
        l_wi += l_pk * 10.0 * kBstar * ki;
        l_ki += l_pk * 10.0 * kBstar * wi;
    }
    l_nti += l_pk0 * Q;
    l_Q += l_pk0 * nti;
    l_dv -= l_pk0 * (2.0 / 3.0) * ki;
    l_ki -= l_pk0 * (2.0 / 3.0) * dv;
    l_f1 += l_gam * (cw1 - cw2);
    double l_SS = 2.0 * l_Q;
    l_dv -= l_Q * (4.0 / 3.0) * dv;
    if (Sabs > 0.0) l_SS += l_Sabs / Sabs;
    l_g[0] += l_SS * 2.0 * s11 + l_dv;
    l_g[3] += l_SS * 2.0 * s22 + l_dv;
    l_g[1] += l_SS * 2.0 * s12;
    l_g[2] += l_SS * 2.0 * s12;
    // faces
    double l_sk = 0.0, l_sw = 0.0;
    for (int m = 0; m < 4; ++m) {
        const SstFace<double> &f = F[m];
        if (!f.has) continue;
        const double kin = ki + lgi[0] * f.rox + lgi[1] * f.roy;
        const double win = wi + lgi[2] * f.rox + lgi[3] * f.roy;
        const double dla = sqrt(f.snx * f.snx + f.sny * f.sny);
        double l_kin = 0, l_win = 0;
        double lf[kSstFU] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // u v k w, lg0..3, f1, nut, gn0..3
        double dkn, dwn;
        sst_face_normal_gradients(f, g, ki, wi, dla, nonorth, dkn, dwn);
        if (!f.bnd) {
            const double un = 0.5 * (ui + f.u) * f.snx + 0.5 * (vi + f.v) * f.sny;
            const bool up = un >= 0.0;
            const double kup = up ? kin : f.k + f.lg[0] * f.rnx + f.lg[1] * f.rny;
            const double wup = up ? win : f.w + f.lg[2] * f.rnx + f.lg[3] * f.rny;
            const double skj = f.f1 * kSk1 + (1.0 - f.f1) * kSk2;
            const double swj = f.f1 * kSw1 + (1.0 - f.f1) * kSw2;
            const double gkf = 0.5 * ((nu + sk_i * nti) + (nu + skj * f.nut));
            const double gwf = 0.5 * ((nu + sw_i * nti) + (nu + swj * f.nut));
            const double l_un = l_ck * kup + l_cw * wup;
            const double l_kup = l_ck * un, l_wup = l_cw * un;
            const double l_gkf = l_dk * dkn * dla, l_gwf = l_dw * dwn * dla;
            const double l_dkn = l_dk * gkf * dla, l_dwn = l_dw * gwf * dla;
            if (nonorth) sst_face_correction_T(f, g, dla, l_dkn, l_dwn, l_g, lf, AG, m, np, i);
            if (AG.sn != nullptr) {  // geometry: n dl / A (through u.n and dl/A), r_nbr, 1/|d|
                const double l_dla = l_dk * gkf * dkn + l_dw * gwf * dwn;
                AG.sn[(2 * m) * np + i] += l_un * 0.5 * (ui + f.u) + l_dla * f.snx / dla;
                AG.sn[(2 * m + 1) * np + i] += l_un * 0.5 * (vi + f.v) + l_dla * f.sny / dla;
                if (!up) {
                    AG.rnbr[(2 * m) * np + i] += l_kup * f.lg[0] + l_wup * f.lg[2];
                    AG.rnbr[(2 * m + 1) * np + i] += l_kup * f.lg[1] + l_wup * f.lg[3];
                }
                AG.dinv[m * np + i] += l_dkn * (f.k - ki) + l_dwn * (f.w - wi);
            }
            lf[2] += l_dkn * f.dinv;
            l_ki -= l_dkn * f.dinv;
            lf[3] += l_dwn * f.dinv;
            l_wi -= l_dwn * f.dinv;
            l_sk += 0.5 * l_gkf * nti;
            l_sw += 0.5 * l_gwf * nti;
            l_nti += 0.5 * (l_gkf * sk_i + l_gwf * sw_i);
            lf[9] += 0.5 * (l_gkf * skj + l_gwf * swj);
            lf[8] += 0.5 * f.nut * (l_gkf * (kSk1 - kSk2) + l_gwf * (kSw1 - kSw2));
            if (up) {
                l_kin += l_kup;
                l_win += l_wup;
            } else {
                lf[2] += l_kup;
                lf[4] += l_kup * f.rnx;
                lf[5] += l_kup * f.rny;
                lf[3] += l_wup;
                lf[6] += l_wup * f.rnx;
                lf[7] += l_wup * f.rny;
            }
            l_ui += 0.5 * l_un * f.snx;
            lf[0] += 0.5 * l_un * f.snx;
            l_vi += 0.5 * l_un * f.sny;
            lf[1] += 0.5 * l_un * f.sny;
        } else {
            const double un = f.u * f.snx + f.v * f.sny;
            const bool up = un >= 0.0;
            const double kup = up ? kin : f.k, wup = up ? win : f.w;
            const double l_un = l_ck * kup + l_cw * wup;
            if (up) {
                l_kin += l_ck * un;
                l_win += l_cw * un;
            } else {
                lf[2] += l_ck * un;
                lf[3] += l_cw * un;
            }
            lf[0] += l_un * f.snx;
            lf[1] += l_un * f.sny;
            if (AG.sn != nullptr) {
                const double l_dla = l_dk * (nu + sk_i * nti) * dkn + l_dw * (nu + sw_i * nti) * dwn;
                AG.sn[(2 * m) * np + i] += l_un * f.u + l_dla * f.snx / dla;
                AG.sn[(2 * m + 1) * np + i] += l_un * f.v + l_dla * f.sny / dla;
                AG.dinv[m * np + i] += l_dk * (nu + sk_i * nti) * dla * (f.k - ki) +
                                       l_dw * (nu + sw_i * nti) * dla * (f.w - wi);
            }
            l_sk += l_dk * nti * dkn * dla;
            l_sw += l_dw * nti * dwn * dla;
            l_nti += (l_dk * sk_i * dkn + l_dw * sw_i * dwn) * dla;
            const double l_dkn = l_dk * (nu + sk_i * nti) * dla, l_dwn = l_dw * (nu + sw_i * nti) * dla;
            if (nonorth) sst_face_correction_T(f, g, dla, l_dkn, l_dwn, l_g, lf, AG, m, np, i);
            lf[2] += l_dkn * f.dinv;
            l_ki -= l_dkn * f.dinv;
            lf[3] += l_dwn * f.dinv;
            l_wi -= l_dwn * f.dinv;
            double lown[4] = {0, 0, 0, 0};
            if (G.btype[-G.nbr[m * np + i] - 1] == FVLBM_BC_WALL)  // omega_b = 60 nu / (beta1 d^2)
                l_di -= lf[3] * 2.0 * f.w / di;
            sst_bvals_T(G, -G.nbr[m * np + i] - 1, lf, lown, lbval);
            l_ui += lown[0];
            l_vi += lown[1];
            l_ki += lown[2];
            l_wi += lown[3];
#pragma unroll
            for (int c = 0; c < kSstFU; ++c) lf[c] = 0.0;  // nothing goes to a neighbour
        }
        if (AG.sn != nullptr) {
            AG.rown[(2 * m) * np + i] += l_kin * lgi[0] + l_win * lgi[2];
            AG.rown[(2 * m + 1) * np + i] += l_kin * lgi[1] + l_win * lgi[3];
        }
        l_ki += l_kin;
        l_lgi[0] += l_kin * f.rox;
        l_lgi[1] += l_kin * f.roy;
        l_wi += l_win;
        l_lgi[2] += l_win * f.rox;
        l_lgi[3] += l_win * f.roy;
#pragma unroll
        for (int c = 0; c < kSstFU; ++c) fbuf[(c * 4 + m) * np + i] = lf[c];
    }
    l_f1 += l_sk * (kSk1 - kSk2) + l_sw * (kSw1 - kSw2);
    if (AG.sn != nullptr) AG.wd[i] += l_di;
    own[0 * np + i] = l_ui;
    own[1 * np + i] = l_vi;
    own[2 * np + i] = l_ki;
    own[3 * np + i] = l_wi;
    own[4 * np + i] = l_nti;
#pragma unroll
    for (int c = 0; c < 8; ++c) own[(5 + c) * np + i] = l_g[c];
#pragma unroll
    for (int c = 0; c < 4; ++c) own[(13 + c) * np + i] = l_lgi[c];
    own[17 * np + i] = l_f1;
}

// ---- reverse of sst_cell_grad of one cell.  The adjoints of its limited gradients and f1 are
// its own (from its update) plus what its neighbours' updates wrote for them; the adjoints of
// (u, v, k, omega) it produces go to its own slots in `own` and to the per-face buffer.
__global__ void __launch_bounds__(kTile) k_adj_sst_grad(
    const double *__restrict__ mac, const double *__restrict__ kk, const double *__restrict__ ww,
    const double *__restrict__ grads, const double *__restrict__ f1a, const double *__restrict__ fbu,
    double *__restrict__ own, double *__restrict__ fbg, double *__restrict__ lbval, Geo<double> G,
    const int *__restrict__ back, AdjGeo AG) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    if (!P.sst) return;
    const double nu = P.nu;
    const double ow[4] = {mac[np + i], mac[2 * np + i], kk[i], ww[i]};
    const double ki = ow[2], wi = ow[3];
    const double di = G.wdist[i];
    double g[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) g[c] = grads[c * np + i];
    // adjoints of lg and f1: own + neighbours' (their face slot facing this cell)
    double l_lg[4], l_f1 = own[17 * np + i], l_g[8];
#pragma unroll
    for (int c = 0; c < 4; ++c) l_lg[c] = own[(13 + c) * np + i];
#pragma unroll
    for (int c = 0; c < 8; ++c) l_g[c] = own[(5 + c) * np + i];
    int nbs[4];
    bool has[4];
    double q[4][4], W[8], R[8];
    for (int m = 0; m < 4; ++m) {
        nbs[m] = G.nbr[m * np + i];
        has[m] = nbs[m] != kNone;
        W[2 * m] = G.lsq[(2 * m) * np + i];
        W[2 * m + 1] = G.lsq[(2 * m + 1) * np + i];
        R[2 * m] = G.rown[(2 * m) * np + i];
        R[2 * m + 1] = G.rown[(2 * m + 1) * np + i];
        const int nb = nbs[m];
        if (nb == kNone) continue;
        if (nb >= 0) {
            q[m][0] = mac[np + nb];
            q[m][1] = mac[2 * np + nb];
            q[m][2] = kk[nb];
            q[m][3] = ww[nb];
            const int b = back[m * np + i];
#pragma unroll
            for (int c = 0; c < 4; ++c) l_lg[c] += fbu[((4 + c) * 4 + b) * np + nb];
            l_f1 += fbu[(8 * 4 + b) * np + nb];
#pragma unroll
            for (int c = 0; c < 4; ++c) l_g[4 + c] += fbu[((10 + c) * 4 + b) * np + nb];
        } else {
            sst_bvals(G, -nb - 1, nu, ow[0], ow[1], ow[2], ow[3], di, q[m][0], q[m][1], q[m][2], q[m][3]);
        }
    }
    // ---------------- forward of the limiters and f1
    double kq[4], wq[4];
    for (int m = 0; m < 4; ++m) {
        kq[m] = has[m] ? ki + (q[m][2] - ki) : ki;
        wq[m] = has[m] ? wi + (q[m][3] - wi) : wi;
    }
    // extremes with the tangent's tie rule (fmin / fmax keep the first argument on ties):
    // index -1 is the cell itself
    double klo = ki, khi = ki, wlo = wi, whi = wi;
    int iklo = -1, ikhi = -1, iwlo = -1, iwhi = -1;
    for (int m = 0; m < 4; ++m) {
        if (kq[m] < klo) { klo = kq[m]; iklo = has[m] ? m : -1; }
        if (kq[m] > khi) { khi = kq[m]; ikhi = has[m] ? m : -1; }
        if (wq[m] < wlo) { wlo = wq[m]; iwlo = has[m] ? m : -1; }
        if (wq[m] > whi) { whi = wq[m]; iwhi = has[m] ? m : -1; }
    }
    double pk = 1.0, pw = 1.0;
    int mk = -1, mw = -1;  // face giving the limiter (-1: none, pk = 1)
    bool khi_side = false, whi_side = false;
    for (int m = 0; m < 4; ++m) {
        if (!has[m]) continue;
        const double rx = R[2 * m], ry = R[2 * m + 1];
        const double dkf = g[4] * rx + g[5] * ry, dwf = g[6] * rx + g[7] * ry;
        if (dkf > 0.0) {
            const double r = (khi - ki) / dkf;
            if (r < pk) { pk = r; mk = m; khi_side = true; }
        } else if (dkf < 0.0) {
            const double r = (klo - ki) / dkf;
            if (r < pk) { pk = r; mk = m; khi_side = false; }
        }
        if (dwf > 0.0) {
            const double r = (whi - wi) / dwf;
            if (r < pw) { pw = r; mw = m; whi_side = true; }
        } else if (dwf < 0.0) {
            const double r = (wlo - wi) / dwf;
            if (r < pw) { pw = r; mw = m; whi_side = false; }
        }
    }
    const double G46 = g[4] * g[6] + g[5] * g[7];
    const double cd0 = 2.0 * kSw2 / wi * G46;
    const double cd = cd0 > 1e-20 ? cd0 : 1e-20;
    const double sk = sqrt(ki);
    const double a = sk / (kBstar * wi * di);
    const double bb = 500.0 * nu / (wi * di * di);
    const double c = 4.0 * kSw2 * ki / (cd * di * di);
    const double M = bb > a ? bb : a;
    const double arg1 = c < M ? c : M;
    const double a2 = arg1 * arg1;
    const double f1 = tanh(a2 * a2);
    // ---------------- reverse
    double l_own[4] = {0, 0, 0, 0};  // u, v, k, omega of this cell
    double l_q[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
    const double l_arg1 = l_f1 * (1.0 - f1 * f1) * 4.0 * arg1 * a2;
    double l_c = 0.0, l_M = 0.0;
    if (c < M) l_c = l_arg1; else l_M = l_arg1;
    double l_a = 0.0, l_bb = 0.0;
    if (bb > a) l_bb = l_M; else l_a = l_M;
    if (sk > 0.0) l_own[2] += l_a * a / (2.0 * ki);
    l_own[3] -= l_a * a / wi;
    l_own[3] -= l_bb * bb / wi;
    l_own[2] += l_c * 4.0 * kSw2 / (cd * di * di);
    double l_di = -(l_a * a + 2.0 * l_bb * bb + 2.0 * l_c * c) / di;
    const double l_cd = -l_c * c / cd;
    if (cd0 > 1e-20) {
        l_own[3] -= l_cd * cd0 / wi;
        const double l_G = l_cd * 2.0 * kSw2 / wi;
        l_g[4] += l_G * g[6];
        l_g[6] += l_G * g[4];
        l_g[5] += l_G * g[7];
        l_g[7] += l_G * g[5];
    }
    const double l_pk = l_lg[0] * g[4] + l_lg[1] * g[5];
    const double l_pw = l_lg[2] * g[6] + l_lg[3] * g[7];
    l_g[4] += l_lg[0] * pk;
    l_g[5] += l_lg[1] * pk;
    l_g[6] += l_lg[2] * pw;
    l_g[7] += l_lg[3] * pw;
    if (mk >= 0) {  // pk = (k_ext - k_i) / (g_k . r_m)
        const double rx = R[2 * mk], ry = R[2 * mk + 1];
        const double dkf = g[4] * rx + g[5] * ry;
        const double l_N = l_pk / dkf, l_d = -l_pk * pk / dkf;
        l_g[4] += l_d * rx;
        l_g[5] += l_d * ry;
        if (AG.sn != nullptr) {
            AG.rown[(2 * mk) * np + i] += l_d * g[4];
            AG.rown[(2 * mk + 1) * np + i] += l_d * g[5];
        }
        const int e = khi_side ? ikhi : iklo;  // the extreme: -1 is k_i itself (k_i - k_i)
        if (e >= 0) {
            l_q[e][2] += l_N;
            l_own[2] -= l_N;
        }
    }
    if (mw >= 0) {
        const double rx = R[2 * mw], ry = R[2 * mw + 1];
        const double dwf = g[6] * rx + g[7] * ry;
        const double l_N = l_pw / dwf, l_d = -l_pw * pw / dwf;
        l_g[6] += l_d * rx;
        l_g[7] += l_d * ry;
        if (AG.sn != nullptr) {
            AG.rown[(2 * mw) * np + i] += l_d * g[6];
            AG.rown[(2 * mw + 1) * np + i] += l_d * g[7];
        }
        const int e = whi_side ? iwhi : iwlo;
        if (e >= 0) {
            l_q[e][3] += l_N;
            l_own[3] -= l_N;
        }
    }
    // g = sum_m W_m (q_m - own)
    for (int m = 0; m < 4; ++m) {
        if (!has[m]) continue;
        double lwx = 0.0, lwy = 0.0;
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
            const double l = W[2 * m] * l_g[2 * c4] + W[2 * m + 1] * l_g[2 * c4 + 1];
            l_q[m][c4] += l;
            l_own[c4] -= l;
            lwx += l_g[2 * c4] * (q[m][c4] - ow[c4]);
            lwy += l_g[2 * c4 + 1] * (q[m][c4] - ow[c4]);
        }
        if (AG.sn != nullptr) {
            AG.lsq[(2 * m) * np + i] += lwx;
            AG.lsq[(2 * m + 1) * np + i] += lwy;
        }
    }
    for (int m = 0; m < 4; ++m) {
        double out[kSstFG] = {0, 0, 0, 0};
        if (has[m]) {
            if (nbs[m] >= 0) {
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) out[c4] = l_q[m][c4];
            } else {
                if (G.btype[-nbs[m] - 1] == FVLBM_BC_WALL) l_di -= l_q[m][3] * 2.0 * q[m][3] / di;
                sst_bvals_T(G, -nbs[m] - 1, l_q[m], l_own, lbval);
            }
        }
#pragma unroll
        for (int c4 = 0; c4 < kSstFG; ++c4) fbg[(c4 * 4 + m) * np + i] = out[c4];
    }
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) own[c4 * np + i] += l_own[c4];
    if (AG.sn != nullptr) AG.wd[i] += l_di;
}

// ---- totals: lam(u, v, k, omega, nu_t) of every cell = own + neighbours' face entries; the
// (u, v) part goes into lam_f through the moments of f^n, (k, omega, nu_t) become the state
// adjoints of the previous step.
__global__ void __launch_bounds__(kTile) k_adj_sst_finish(
    const double *__restrict__ fn, const double *__restrict__ own, const double *__restrict__ fbu,
    const double *__restrict__ fbg, double *__restrict__ lf, double *__restrict__ lk,
    double *__restrict__ lw, double *__restrict__ lnt, Geo<double> G, const int *__restrict__ back, bool add) {
    const int i = blockIdx.x * kTile + threadIdx.x;
    const size_t np = G.np;
    const InstParam P = G.ip[G.tile_inst[blockIdx.x]];
    if (!P.sst) return;
    double l[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) l[c] = own[c * np + i];
    for (int m = 0; m < 4; ++m) {
        const int nb = G.nbr[m * np + i];
        if (nb < 0) continue;
        const int b = back[m * np + i];
#pragma unroll
        for (int c = 0; c < 4; ++c) l[c] += fbu[(c * 4 + b) * np + nb] + fbg[(c * 4 + b) * np + nb];
        l[4] += fbu[(9 * 4 + b) * np + nb];
    }
    if (add) {  // several solves read the same state (per-stage reading)
        lk[i] += l[2];
        lw[i] += l[3];
        lnt[i] += l[4];
    } else {
        lk[i] = l[2];
        lw[i] = l[3];
        lnt[i] = l[4];
    }
    double f[kQ], dr, r, u, v, lfi[kQ];
    load9(fn, np, i, f);
    moments(f, P.rho0, dr, r, u, v);
#pragma unroll
    for (int a = 0; a < kQ; ++a) lfi[a] = lf[a * np + i];
    moments_vjp(r, u, v, 0.0, l[0], l[1], lfi);
#pragma unroll
    for (int a = 0; a < kQ; ++a) lf[a * np + i] = lfi[a];
}

}  // namespace fvlbm
