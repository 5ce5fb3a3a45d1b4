// Reverse-mode derivatives of the per-node pieces of the LBM step (the
// adjoint of the method for gradients of a wall force with respect to the
// geometry), written by hand from the forward arithmetic of step_core,
// boundary_pops, k_wall_force, the rest initialisation and k_metric.
//
// Conventions: every function recomputes the forward intermediates it needs
// from the same inputs as the forward pass, then propagates adjoints (the
// "l" prefix) from outputs to inputs.  Symmetric 3x3 tensors are packed as
// (00, 01, 02, 11, 12, 22); the adjoint of a packed entry is the derivative
// with respect to that stored value (an off-diagonal value stands for both
// (a, b) and (b, a)).  The geometry adjoint of a node has the layout of its
// geometry: [0] sqrt(g), [1..6] g^ij, [7..24] Gamma^i_jk at i*6 + s6(j,k).
#pragma once

#include "flat_step.cuh"

namespace cslbm {
namespace adj {

constexpr int NG = 25;

// the weight of packed entry k in c c : E  (c_a^2 on the diagonal, 2 c_a c_b off it)
__device__ __forceinline__ constexpr int cmul(int l, int k)
{
    return k == 0 ? cvec(l, 0) * cvec(l, 0)
         : k == 3 ? cvec(l, 1) * cvec(l, 1)
         : k == 5 ? cvec(l, 2) * cvec(l, 2)
         : k == 1 ? 2 * cvec(l, 0) * cvec(l, 1)
         : k == 2 ? 2 * cvec(l, 0) * cvec(l, 2)
                  : 2 * cvec(l, 1) * cvec(l, 2);
}
__device__ __forceinline__ constexpr int ka(int k) { return k == 0 || k == 1 || k == 2 ? 0 : (k == 5 ? 2 : 1); }
__device__ __forceinline__ constexpr int kb(int k) { return k == 0 ? 0 : k == 1 || k == 3 ? 1 : 2; }
__device__ __forceinline__ constexpr bool kdiag(int k) { return k == 0 || k == 3 || k == 5; }

template <class R> struct Moms {
    R m0, m1[3], m2[6];
};
template <class R> __device__ __forceinline__ void moments_of(const R s[Q], Moms<R>& M)
{
    M.m0 = R(0);
#pragma unroll
    for (int a = 0; a < 3; a++) M.m1[a] = R(0);
#pragma unroll
    for (int k = 0; k < 6; k++) M.m2[k] = R(0);
#pragma unroll
    for (int l = 0; l < Q; l++) {
        M.m0 += s[l];
#pragma unroll
        for (int a = 0; a < 3; a++) M.m1[a] += R(cvec(l, a)) * s[l];
#pragma unroll
        for (int k = 0; k < 6; k++) M.m2[k] += R(cvec(l, ka(k)) * cvec(l, kb(k))) * s[l];
    }
}
// adjoint of the moments onto the populations
template <class R>
__device__ __forceinline__ void moments_reverse(const R lm0, const R lm1[3], const R lm2[6], R ls[Q])
{
#pragma unroll
    for (int l = 0; l < Q; l++) {
        R v = lm0;
#pragma unroll
        for (int a = 0; a < 3; a++) v += R(cvec(l, a)) * lm1[a];
#pragma unroll
        for (int k = 0; k < 6; k++) v += R(cvec(l, ka(k)) * cvec(l, kb(k))) * lm2[k];
        ls[l] += v;
    }
}

// ---------------------------------------------------------------------------
// the step of an interior node (step_core): inputs s (pulled, shifted), the
// geometry G, the history Hp at time t and the nine rho-u differences d;
// outputs the post-collision populations and the new history.  Given the
// adjoints lout, lH of the outputs, accumulates the adjoints of s (ls), of
// Hp (lHp), of the geometry (lgeo) and of the lattice gradient D (lD).
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void step_reverse(const Lat& L, const R s[Q], const GeoT<R>& G, const HistT<R>& Hp,
                                             const R d[9][3], const R lout[Q], const HistT<R>& lH, R ls[Q],
                                             HistT<R>& lHp, R lgeo[NG], R lD[3][3])
{
    const R th = R(L.theta), kv = R(L.kvisc), om = R(L.omega), cs2 = R(1.0 / 3.0);
    // ---- forward ----
    Moms<R> M;
    moments_of(s, M);
    const R sg = G.sg, isg = R(1) / sg;
    const R rho = sg * (M.m0 + R(1)) + R(0.5) * Hp.A, ir = R(1) / rho;
    R j[3];
#pragma unroll
    for (int a = 0; a < 3; a++) j[a] = sg * M.m1[a] + R(0.5) * Hp.B[a];
    const R rt = rho * th;
    R pieq[6], pi[6], T[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        pieq[k] = j[ka(k)] * j[kb(k)] * ir + rt * G.gi[k];
        pi[k] = sg * (M.m2[k] + (kdiag(k) ? cs2 : R(0))) + R(0.5) * Hp.C[k];
        T[k] = kv * (pi[k] - pieq[k]) + pieq[k];
    }
    R gc[3];
#pragma unroll
    for (int k = 0; k < 3; k++) gc[k] = G.gam[0 * 6 + s6(k, 0)] + G.gam[1 * 6 + s6(k, 1)] + G.gam[2 * 6 + s6(k, 2)];
    R D[3][3];
    gradient_from_pairs(d, D);
    R A = R(0);
#pragma unroll
    for (int k = 0; k < 3; k++) A -= R(2) * gc[k] * j[k];
    R B[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        R g = R(0), gt = R(0);
#pragma unroll
        for (int k = 0; k < 6; k++) g += G.gam[i * 6 + k] * T[k] * R(kdiag(k) ? 1 : 2);
#pragma unroll
        for (int jj = 0; jj < 3; jj++) gt += gc[jj] * T[s6(i, jj)];
        B[i] = R(L.fext[i]) - g - R(2) * gt;
    }
    R bard[3][3], cov[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int i = 0; i < 3; i++) {
            bard[k][i] = D[k][i] - gc[k] * j[i];
            R c = D[k][i];
#pragma unroll
            for (int l = 0; l < 3; l++) c += G.gam[i * 6 + s6(k, l)] * j[l];
            cov[k][i] = c;
        }
    const R divcov = cov[0][0] + cov[1][1] + cov[2][2];
    R C[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int i = ka(k), jj = kb(k);
        R c = bard[jj][i] + bard[i][jj];
        if (i == jj) c += bard[0][0] + bard[1][1] + bard[2][2];
        R t = G.gi[k] * divcov;
#pragma unroll
        for (int q = 0; q < 3; q++) t += G.gi[s6(jj, q)] * cov[q][i] + G.gi[s6(i, q)] * cov[q][jj];
        C[k] = cs2 * c - th * t;
    }
    R E1[3], E2[6];
#pragma unroll
    for (int a = 0; a < 3; a++) E1[a] = om * j[a] + B[a] - R(0.5) * om * Hp.B[a];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const R a2 = j[ka(k)] * j[kb(k)] * ir + rt * G.gi[k] - (kdiag(k) ? rho * cs2 : R(0));
        const R b2 = C[k] - (kdiag(k) ? A * cs2 : R(0));
        const R b2p = Hp.C[k] - (kdiag(k) ? Hp.A * cs2 : R(0));
        E2[k] = om * a2 + b2 - R(0.5) * om * b2p;
    }
    const R d0 = om * M.m0 + A * isg;
    const R tE = R(1.5) * (E2[0] + E2[3] + E2[5]);

    // ---- reverse ----
    R lisg = R(0), lsg = R(0), lrho = R(0), lir = R(0), lm0 = R(0), lj[3] = {0, 0, 0}, lm1[3] = {0, 0, 0};
    R lm2[6] = {0, 0, 0, 0, 0, 0}, lT[6] = {0, 0, 0, 0, 0, 0}, lgc[3] = {0, 0, 0};
    R lA = lH.A, lB[3] = {lH.B[0], lH.B[1], lH.B[2]}, lC[6];
#pragma unroll
    for (int k = 0; k < 6; k++) lC[k] = lH.C[k];
    // collision
    R ld0 = R(0), lE1[3] = {0, 0, 0}, lE2[6] = {0, 0, 0, 0, 0, 0}, ltE = R(0);
#pragma unroll
    for (int l = 0; l < Q; l++) {
        const R w = R(wq(l)), q = w * lout[l];
        ls[l] += (R(1) - om) * lout[l];
        ld0 += q;
        R e1c = R(0), e2c = R(0);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            e1c += E1[a] * R(cvec(l, a));
            lE1[a] += R(3) * isg * q * R(cvec(l, a));
        }
#pragma unroll
        for (int k = 0; k < 6; k++) {
            e2c += E2[k] * R(cmul(l, k));
            lE2[k] += R(4.5) * isg * q * R(cmul(l, k));
        }
        lisg += q * (R(3) * e1c + R(4.5) * e2c - tE);
        ltE -= isg * q;
    }
    lE2[0] += R(1.5) * ltE;
    lE2[3] += R(1.5) * ltE;
    lE2[5] += R(1.5) * ltE;
    lm0 += om * ld0;
    lA += isg * ld0;
    lisg += A * ld0;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const R la2 = om * lE2[k], lb2 = lE2[k], lb2p = R(-0.5) * om * lE2[k];
        lC[k] += lb2;
        lHp.C[k] += lb2p;
        if (kdiag(k)) {
            lA -= cs2 * lb2;
            lHp.A -= cs2 * lb2p;
            lrho -= cs2 * la2;
        }
        // a2 = j_a j_b ir + rho theta g^ab
        lj[ka(k)] += la2 * j[kb(k)] * ir;
        lj[kb(k)] += la2 * j[ka(k)] * ir;
        lir += la2 * j[ka(k)] * j[kb(k)];
        lrho += la2 * th * G.gi[k];
        lgeo[1 + k] += la2 * rt;
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lj[a] += om * lE1[a];
        lB[a] += lE1[a];
        lHp.B[a] += R(-0.5) * om * lE1[a];
    }
    // forcing moment C
    R lbard[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, lcov[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    R ldivbar = R(0), ldivcov = R(0);
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int i = ka(k), jj = kb(k);
        const R lc = cs2 * lC[k], lt = -th * lC[k];
        lbard[jj][i] += lc;
        lbard[i][jj] += lc;
        if (i == jj) ldivbar += lc;
        lgeo[1 + k] += lt * divcov;
        ldivcov += lt * G.gi[k];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            lgeo[1 + s6(jj, q)] += lt * cov[q][i];
            lcov[q][i] += lt * G.gi[s6(jj, q)];
            lgeo[1 + s6(i, q)] += lt * cov[q][jj];
            lcov[q][jj] += lt * G.gi[s6(i, q)];
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        lbard[k][k] += ldivbar;
        lcov[k][k] += ldivcov;
    }
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int i = 0; i < 3; i++) {
            lD[k][i] += lbard[k][i] + lcov[k][i];
            lgc[k] -= lbard[k][i] * j[i];
            lj[i] -= lbard[k][i] * gc[k];
#pragma unroll
            for (int l = 0; l < 3; l++) {
                lgeo[7 + i * 6 + s6(k, l)] += lcov[k][i] * j[l];
                lj[l] += lcov[k][i] * G.gam[i * 6 + s6(k, l)];
            }
        }
    // forcing moment B
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const R lg = -lB[i], lgt = R(-2) * lB[i];
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const R m = R(kdiag(k) ? 1 : 2);
            lgeo[7 + i * 6 + k] += lg * T[k] * m;
            lT[k] += lg * G.gam[i * 6 + k] * m;
        }
#pragma unroll
        for (int jj = 0; jj < 3; jj++) {
            lgc[jj] += lgt * T[s6(i, jj)];
            lT[s6(i, jj)] += lgt * gc[jj];
        }
    }
    // forcing moment A
#pragma unroll
    for (int k = 0; k < 3; k++) {
        lgc[k] -= R(2) * j[k] * lA;
        lj[k] -= R(2) * gc[k] * lA;
    }
    // contracted symbol
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int i = 0; i < 3; i++) lgeo[7 + i * 6 + s6(k, i)] += lgc[k];
    // stress
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const R lpi = kv * lT[k], lpe = (R(1) - kv) * lT[k];
        lsg += lpi * (M.m2[k] + (kdiag(k) ? cs2 : R(0)));
        lm2[k] += lpi * sg;
        lHp.C[k] += R(0.5) * lpi;
        lj[ka(k)] += lpe * j[kb(k)] * ir;
        lj[kb(k)] += lpe * j[ka(k)] * ir;
        lir += lpe * j[ka(k)] * j[kb(k)];
        lrho += lpe * th * G.gi[k];
        lgeo[1 + k] += lpe * rt;
    }
    // moments
    lrho -= ir * ir * lir;
    lsg += (M.m0 + R(1)) * lrho;
    lm0 += sg * lrho;
    lHp.A += R(0.5) * lrho;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lsg += M.m1[a] * lj[a];
        lm1[a] += sg * lj[a];
        lHp.B[a] += R(0.5) * lj[a];
    }
    lsg -= isg * isg * lisg;
    lgeo[0] += lsg;
    moments_reverse(lm0, lm1, lm2, ls);
}

// adjoint of D = gradient_from_pairs(d) onto d
template <class R> __device__ __forceinline__ void gradient_reverse(const R lD[3][3], R ld[9][3])
{
    const R wf(1.0 / 6.0), we(1.0 / 12.0);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        ld[0][i] = wf * lD[0][i];
        ld[1][i] = wf * lD[1][i];
        ld[2][i] = wf * lD[2][i];
        ld[3][i] = we * (lD[0][i] + lD[1][i]);
        ld[4][i] = we * (lD[0][i] - lD[1][i]);
        ld[5][i] = we * (lD[0][i] + lD[2][i]);
        ld[6][i] = we * (lD[0][i] - lD[2][i]);
        ld[7][i] = we * (lD[1][i] + lD[2][i]);
        ld[8][i] = we * (lD[1][i] - lD[2][i]);
    }
}

// ---------------------------------------------------------------------------
// Hermite recomposition h_l = w_l isg (b0 + 3 b1.c + 4.5 b2:cc - 1.5 tr b2)
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void hermite_reverse(int l, R isg, R b0, const R b1[3], const R b2[6], R lh, R& lisg,
                                                R& lb0, R lb1[3], R lb2[6])
{
    const R w = R(wq(l));
    R v = b0 - R(1.5) * (b2[0] + b2[3] + b2[5]);
#pragma unroll
    for (int a = 0; a < 3; a++) v += R(3) * b1[a] * R(cvec(l, a));
#pragma unroll
    for (int k = 0; k < 6; k++) v += R(4.5) * b2[k] * R(cmul(l, k));
    lisg += w * v * lh;
    const R q = w * isg * lh;
    lb0 += q;
#pragma unroll
    for (int a = 0; a < 3; a++) lb1[a] += R(3) * R(cvec(l, a)) * q;
#pragma unroll
    for (int k = 0; k < 6; k++) lb2[k] += (R(4.5) * R(cmul(l, k)) - (kdiag(k) ? R(1.5) : R(0))) * q;
}

// forcing term F_l(isg, H): b0 = A, b1 = B, b2 = C - delta A / 3
template <class R>
__device__ __forceinline__ void forcing_reverse(int l, R isg, const Hist<R>& H, R lf, R& lisg, Hist<R>& lHh)
{
    R b2[6];
#pragma unroll
    for (int k = 0; k < 6; k++) b2[k] = H.C[k] - (kdiag(k) ? H.A * R(1.0 / 3.0) : R(0));
    R lb0 = R(0), lb1[3] = {0, 0, 0}, lb2[6] = {0, 0, 0, 0, 0, 0};
    hermite_reverse(l, isg, H.A, H.B, b2, lf, lisg, lb0, lb1, lb2);
    lHh.A += lb0 - R(1.0 / 3.0) * (lb2[0] + lb2[3] + lb2[5]);
#pragma unroll
    for (int a = 0; a < 3; a++) lHh.B[a] += lb1[a];
#pragma unroll
    for (int k = 0; k < 6; k++) lHh.C[k] += lb2[k];
}

// a2 = feq_coeffs(rho, j, gi): adjoint onto rho, j, gi
template <class R>
__device__ __forceinline__ void feq_coeffs_reverse(R rho, const R j[3], const R gi[6], R th, const R la2[6], R& lrho,
                                                   R lj[3], R lgi[6])
{
    const R ir = R(1) / rho;
    R lir = R(0);
#pragma unroll
    for (int k = 0; k < 6; k++) {
        lrho += la2[k] * (th * gi[k] - (kdiag(k) ? R(1.0 / 3.0) : R(0)));
        lgi[k] += la2[k] * rho * th;
        lj[ka(k)] += la2[k] * j[kb(k)] * ir;
        lj[kb(k)] += la2[k] * j[ka(k)] * ir;
        lir += la2[k] * j[ka(k)] * j[kb(k)];
    }
    lrho -= ir * ir * lir;
}

// ---------------------------------------------------------------------------
// boundary rule (boundary_pops) of face node w with inner node i: given the
// adjoint ls of the node's populations, the adjoints of the inner node's
// pulled populations (lsi), of both nodes' sqrt(g) and g^ij (lgi_* with
// [0] = sqrt(g)), and of both histories.  The boundary velocity is a
// constant of the problem.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void boundary_reverse(const Lat& L, int bc, const R si[Q], const Geo<R>& Gi,
                                                 const Geo<R>& Gw, const Hist<R>& Hi, const Hist<R>& Hw,
                                                 const R uw[3], const R ls[Q], R lsi[Q], R lgi_i[7], R lgi_w[7],
                                                 Hist<R>& lHi, Hist<R>& lHw)
{
    const R th = R(L.theta);
    const R ratio = Gi.sg * Gw.isg;
    R lisg_i = R(0), lisg_w = R(0), lratio = R(0);
    R fi[Q];
#pragma unroll
    for (int l = 0; l < Q; l++) fi[l] = si[l] + R(wq(l)) + R(0.5) * forcing_l(l, Gi.isg, Hi);
    // s_l = fw_l - F_l(isg_w, Hw)/2 - w_l
#pragma unroll
    for (int l = 0; l < Q; l++) forcing_reverse(l, Gw.isg, Hw, R(-0.5) * ls[l], lisg_w, lHw);
    R lfi[Q];
    if (bc == BC_OUTFLOW) {
#pragma unroll
        for (int l = 0; l < Q; l++) {
            lfi[l] = ratio * ls[l];
            lratio += fi[l] * ls[l];
        }
    } else {
        Moms<R> M;
        moments_of(si, M);
        const R rho = Gi.sg * (R(1) + M.m0) + R(0.5) * Hi.A;
        R j[3], jw[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            j[a] = Gi.sg * M.m1[a] + R(0.5) * Hi.B[a];
            jw[a] = rho * uw[a];
        }
        R a2w[6], a2i[6];
        feq_coeffs(rho, jw, Gw.gi, th, a2w);
        feq_coeffs(rho, j, Gi.gi, th, a2i);
        R lrho = R(0), lj[3] = {0, 0, 0}, ljw[3] = {0, 0, 0}, la2w[6] = {0, 0, 0, 0, 0, 0},
          la2i[6] = {0, 0, 0, 0, 0, 0};
        R ltmp = R(0);
#pragma unroll
        for (int l = 0; l < Q; l++) {
            // fw = few + (fi - fei) ratio
            const R fei = hermite_l(l, Gi.isg, rho, j, a2i, a2i[0] + a2i[3] + a2i[5]);
            lfi[l] = ratio * ls[l];
            lratio += (fi[l] - fei) * ls[l];
            hermite_reverse(l, Gw.isg, rho, jw, a2w, ls[l], lisg_w, lrho, ljw, la2w);
            hermite_reverse(l, Gi.isg, rho, j, a2i, -ratio * ls[l], lisg_i, ltmp, lj, la2i);
        }
        lrho += ltmp;
        feq_coeffs_reverse(rho, jw, Gw.gi, th, la2w, lrho, ljw, lgi_w + 1);
        feq_coeffs_reverse(rho, j, Gi.gi, th, la2i, lrho, lj, lgi_i + 1);
#pragma unroll
        for (int a = 0; a < 3; a++) lrho += uw[a] * ljw[a];
        // rho, j from the inner node's populations
        lgi_i[0] += (R(1) + M.m0) * lrho;
        lHi.A += R(0.5) * lrho;
        R lm1[3], lm2[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            lgi_i[0] += M.m1[a] * lj[a];
            lm1[a] = Gi.sg * lj[a];
            lHi.B[a] += R(0.5) * lj[a];
        }
        moments_reverse(Gi.sg * lrho, lm1, lm2, lsi);
    }
    // fi = si + w + F_l(isg_i, Hi)/2
#pragma unroll
    for (int l = 0; l < Q; l++) {
        lsi[l] += lfi[l];
        forcing_reverse(l, Gi.isg, Hi, R(0.5) * lfi[l], lisg_i, lHi);
    }
    // ratio = sg_i isg_w; isg = 1/sg
    lgi_i[0] += Gw.isg * lratio;
    lisg_w += Gi.sg * lratio;
    lgi_i[0] -= Gi.isg * Gi.isg * lisg_i;
    lgi_w[0] -= Gw.isg * Gw.isg * lisg_w;
}

// ---------------------------------------------------------------------------
// rest initialisation of a node (rho = 1, u = 0): shifted populations
// s0_l = w_l isg (1 + 4.5 a2:cc - 1.5 tr a2 - 1.5 B0.c) - w_l with
// a2 = theta g^ij - delta/3 and the history (0, B0, 0),
// B0_i = F_i - theta (Gamma^i_jk g^jk + 2 gc_j g^ij).  Adjoint onto the geometry.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void init_reverse(const Lat& L, const GeoT<R>& G, const R ls0[Q], const R lB0h[3],
                                             R lgeo[NG])
{
    const R th = R(L.theta), isg = R(1) / G.sg;
    R a2[6], gc[3], B0[3];
#pragma unroll
    for (int k = 0; k < 6; k++) a2[k] = th * G.gi[k] - (kdiag(k) ? R(1.0 / 3.0) : R(0));
#pragma unroll
    for (int k = 0; k < 3; k++) gc[k] = G.gam[0 * 6 + s6(k, 0)] + G.gam[1 * 6 + s6(k, 1)] + G.gam[2 * 6 + s6(k, 2)];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        R g = R(0), gt = R(0);
#pragma unroll
        for (int k = 0; k < 6; k++) g += G.gam[i * 6 + k] * G.gi[k] * R(kdiag(k) ? 1 : 2);
#pragma unroll
        for (int jj = 0; jj < 3; jj++) gt += gc[jj] * G.gi[s6(i, jj)];
        B0[i] = R(L.fext[i]) - th * (g + R(2) * gt);
    }
    R lisg = R(0), la2[6] = {0, 0, 0, 0, 0, 0}, lB0[3] = {lB0h[0], lB0h[1], lB0h[2]};
#pragma unroll
    for (int l = 0; l < Q; l++) {
        const R q = R(wq(l)) * ls0[l];
        R v = R(1) - R(1.5) * (a2[0] + a2[3] + a2[5]);
#pragma unroll
        for (int k = 0; k < 6; k++) v += R(4.5) * a2[k] * R(cmul(l, k));
#pragma unroll
        for (int a = 0; a < 3; a++) v -= R(1.5) * B0[a] * R(cvec(l, a));
        lisg += q * v;
#pragma unroll
        for (int k = 0; k < 6; k++) la2[k] += isg * q * (R(4.5) * R(cmul(l, k)) - (kdiag(k) ? R(1.5) : R(0)));
#pragma unroll
        for (int a = 0; a < 3; a++) lB0[a] -= R(1.5) * isg * q * R(cvec(l, a));
    }
#pragma unroll
    for (int k = 0; k < 6; k++) lgeo[1 + k] += th * la2[k];
    R lgc[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const R lg = -th * lB0[i], lgt = R(-2) * th * lB0[i];
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const R m = R(kdiag(k) ? 1 : 2);
            lgeo[7 + i * 6 + k] += lg * G.gi[k] * m;
            lgeo[1 + k] += lg * G.gam[i * 6 + k] * m;
        }
#pragma unroll
        for (int jj = 0; jj < 3; jj++) {
            lgc[jj] += lgt * G.gi[s6(i, jj)];
            lgeo[1 + s6(i, jj)] += lgt * gc[jj];
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int i = 0; i < 3; i++) lgeo[7 + i * 6 + s6(k, i)] += lgc[k];
    lgeo[0] -= isg * isg * lisg;
}

// ---------------------------------------------------------------------------
// geometry from the metric (k_metric), FP64: sqrt(det g), g^-1 and
// Gamma^i_jk = 1/2 g^il (d_j g_kl + d_k g_jl - d_l g_jk).  Adjoint of the
// geometry lgeo onto g (lg6) and its derivatives (ldg18, [k][s6]).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void metric_reverse(const double g6[6], const double dg[3][6], const double lgeo[NG],
                                               double lg6[6], double ldg[3][6])
{
    double G[3][3], GI[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) G[a][b] = g6[s6(a, b)];
    const double c00 = G[1][1] * G[2][2] - G[1][2] * G[2][1], c01 = G[1][2] * G[2][0] - G[1][0] * G[2][2],
                 c02 = G[1][0] * G[2][1] - G[1][1] * G[2][0];
    const double det = G[0][0] * c00 + G[0][1] * c01 + G[0][2] * c02, id = 1.0 / det, sd = sqrt(det);
    GI[0][0] = c00 * id;
    GI[1][0] = c01 * id;
    GI[2][0] = c02 * id;
    GI[0][1] = (G[0][2] * G[2][1] - G[0][1] * G[2][2]) * id;
    GI[1][1] = (G[0][0] * G[2][2] - G[0][2] * G[2][0]) * id;
    GI[2][1] = (G[0][1] * G[2][0] - G[0][0] * G[2][1]) * id;
    GI[0][2] = (G[0][1] * G[1][2] - G[0][2] * G[1][1]) * id;
    GI[1][2] = (G[0][2] * G[1][0] - G[0][0] * G[1][2]) * id;
    GI[2][2] = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) * id;
    // Gamma^i_jk = 1/2 sum_l GI[i][l] S_jkl, S_jkl = dg[j][kl] + dg[k][jl] - dg[l][jk]
    double lGI[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int k = 0; k < 6; k++) ldg[0][k] = ldg[1][k] = ldg[2][k] = 0.0;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int p = 0; p < 6; p++) {
            const int jj = ka(p), kk = kb(p);
            const double lgam = lgeo[7 + i * 6 + p];
#pragma unroll
            for (int l = 0; l < 3; l++) {
                const double S = dg[jj][s6(kk, l)] + dg[kk][s6(jj, l)] - dg[l][s6(jj, kk)];
                lGI[i][l] += 0.5 * lgam * S;
                const double t = 0.5 * lgam * GI[i][l];
                ldg[jj][s6(kk, l)] += t;
                ldg[kk][s6(jj, l)] += t;
                ldg[l][s6(jj, kk)] -= t;
            }
        }
    // packed g^ij entries: the stored value equals GI[a][b] (a <= b)
#pragma unroll
    for (int k = 0; k < 6; k++) lGI[ka(k)][kb(k)] += lgeo[1 + k];
    // d GI = -GI dG GI; d sqrt(det) = sqrt(det)/2 GI : dG
    double lG[3][3];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int d = 0; d < 3; d++) {
            double v = 0.5 * sd * GI[c][d] * lgeo[0];
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) v -= GI[a][c] * lGI[a][b] * GI[d][b];
            lG[c][d] = v;
        }
#pragma unroll
    for (int k = 0; k < 6; k++) lg6[k] = kdiag(k) ? lG[ka(k)][kb(k)] : lG[ka(k)][kb(k)] + lG[kb(k)][ka(k)];
}

}  // namespace adj
}  // namespace cslbm
