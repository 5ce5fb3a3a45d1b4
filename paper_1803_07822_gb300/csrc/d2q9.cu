// The two-dimensional (D2Q9) curved-space lattice Boltzmann step (the 2-D
// flag simulations of the paper run the method on D2Q9), with its own small
// C ABI (cslbm2d_*, include/cslbm.h).
//
// Same method and readings as the three-dimensional library: second-order
// Hermite equilibrium with the metric (App. B), forcing moments A, B^i, C^ij
// (Eqs. forcing-A/B/C) with the trapezoidal history, the isotropic gradient
// of App. D over the eight neighbours, non-equilibrium extrapolation at walls
// and inlets, zero-gradient outlets (inner node one step inward along every
// non-periodic face normal, wall > inflow > outflow), the node-wise chart
// change (Sec. IV.B).
//
// State (pull slots, h-form): slot (l, v) holds the post-collision value of
// node v for direction l less the weight w_l, so that a node pulls
// h_l = slot(l, v - c_l) = f_l - w_l - F_l(t - dt)/2 (small numbers near
// rest, which FP32 keeps to more digits); the node's stored forcing
// coefficients A, B, C are the history F(t - dt), whose moments enter rho,
// j and Pi in closed form.  So one step is two kernels: rho u of every node
// (the gradient stencil needs it), then the step of every node into the
// other buffers.
// One thread per node; R = float (FP32 storage and arithmetic) or double.
#include <cstdint>
#include <cstring>
#include <string>

#include "../../include/cslbm.h"

cslbm_status cslbm_record_error(cslbm_status s, const char* msg);

namespace cslbm2d {

constexpr int Q = 9, TB = 256;
enum { PER = 0, WALL = 1, INFLOW = 2, OUTFLOW = 3 };

__host__ __device__ __forceinline__ constexpr int cx(int l)
{
    return l == 1 || l == 5 || l == 7 ? 1 : (l == 2 || l == 6 || l == 8 ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int cy(int l)
{
    return l == 3 || l == 5 || l == 8 ? 1 : (l == 4 || l == 6 || l == 7 ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr double wq(int l)
{
    return l == 0 ? 4.0 / 9.0 : (l <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// geometry per node (10 values): sqrt(g), g^00, g^01, g^11, Gamma^0_{00,01,11}, Gamma^1_{00,01,11}
// forcing coefficients per node: A, B^0, B^1, C^00, C^01, C^11
constexpr int NF = 6;

struct Lat {
    int n[2], lo[2], hi[2];
    long long N;
    double omega, kvisc, theta, fext[2];
    const double* face[4];  // [2][n other] contravariant face velocity, or null
};

template <class R> struct Geo {
    R sg, isg, gi[3], gam[2][3];
};

template <class R> __device__ __forceinline__ void load_geo(const R* __restrict__ G, long long N, long long v, Geo<R>& g)
{
    g.sg = G[v];
    g.isg = R(1) / g.sg;
#pragma unroll
    for (int k = 0; k < 3; k++) g.gi[k] = G[(1 + k) * N + v];
#pragma unroll
    for (int k = 0; k < 6; k++) g.gam[k / 3][k % 3] = G[(4 + k) * N + v];
}

// symmetric 2 x 2 stored as 00, 01, 11
__device__ __forceinline__ int s3(int i, int j) { return i + j; }

// w_l / sqrt(g) (a0 + a1.c / c_s^2 + a2 : (c c - c_s^2 delta) / (2 c_s^4)), c_s^2 = 1/3
template <class R>
__device__ __forceinline__ R hermite(int l, R isg, R a0, const R a1[2], const R a2[3])
{
    const R c0 = R(cx(l)), c1 = R(cy(l));
    const R h1 = a1[0] * c0 + a1[1] * c1;
    const R tr = a2[0] + a2[2];
    const R h2 = a2[0] * c0 * c0 + R(2) * a2[1] * c0 * c1 + a2[2] * c1 * c1 - tr * R(1.0 / 3.0);
    return R(wq(l)) * isg * (a0 + R(3) * h1 + R(4.5) * h2);
}

// F_l from A, B, C: b_(2) = C - c_s^2 delta A
template <class R> __device__ __forceinline__ R forcing_l(int l, R isg, const R Fc[NF])
{
    const R b1[2] = {Fc[1], Fc[2]};
    const R b2[3] = {Fc[3] - Fc[0] * R(1.0 / 3.0), Fc[4], Fc[5] - Fc[0] * R(1.0 / 3.0)};
    return hermite<R>(l, isg, Fc[0], b1, b2);
}

template <class R> __device__ __forceinline__ void feq_all(const Geo<R>& g, R theta, R rho, const R j[2], R out[Q])
{
    const R ir = R(1) / rho;
    R a2[3];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = i; k < 2; k++)
            a2[s3(i, k)] = rho * (theta * g.gi[s3(i, k)] - (i == k ? R(1.0 / 3.0) : R(0))) + j[i] * j[k] * ir;
    // f^eq - w: rho - sqrt(g) in place of rho (w_l / sqrt(g) sqrt(g) = w_l)
    const R a0 = rho - g.sg;
#pragma unroll
    for (int l = 0; l < Q; l++) out[l] = hermite<R>(l, g.isg, a0, j, a2);
}

__device__ __forceinline__ bool wrap(const Lat& L, int a, int& r)
{
    if (r < 0) {
        if (L.lo[a] != PER) return false;
        r += L.n[a];
    } else if (r >= L.n[a]) {
        if (L.hi[a] != PER) return false;
        r -= L.n[a];
    }
    return true;
}

template <class R> __device__ __forceinline__ void load_fc(const R* __restrict__ Fc, long long N, long long v, R out[NF])
{
#pragma unroll
    for (int k = 0; k < NF; k++) out[k] = Fc[k * N + v];
}

// h of an interior node: the pulled slots, h_l = slot (l, x - c_l) =
// f_l - w_l - F_l(t - dt)/2 (periodic wrap at most)
template <class R>
__device__ __forceinline__ void gather_h(const Lat& L, const R* __restrict__ P, int x, int y, R h[Q])
{
    const long long N = L.N;
#pragma unroll
    for (int l = 0; l < Q; l++) {
        int xs = x - cx(l), ys = y - cy(l);
        wrap(L, 0, xs);
        wrap(L, 1, ys);
        h[l] = P[l * N + xs + (long long)L.n[0] * ys];
    }
}

// s = f - w of an interior node: h + F(t - dt)/2 of the node
template <class R>
__device__ __forceinline__ void gather(const Lat& L, const R* __restrict__ P, const R* __restrict__ Fc,
                                       const R* __restrict__ G, int x, int y, R f[Q])
{
    const long long v = x + (long long)L.n[0] * y;
    R fc[NF];
    load_fc(Fc, L.N, v, fc);
    const R isg = R(1) / G[v];
    gather_h<R>(L, P, x, y, f);
#pragma unroll
    for (int l = 0; l < Q; l++) f[l] += R(0.5) * forcing_l<R>(l, isg, fc);
}

// moments of f from s = f - w: rho = sqrt(g)(1 + sum s), j = sqrt(g) sum s c,
// Pi = sqrt(g)(sum s c c + delta / 3) (sum w = 1, sum w c = 0, sum w c c = delta / 3)
template <class R> __device__ __forceinline__ void moments(const R f[Q], R sg, R& rho, R j[2], R Pi[3])
{
    R m0 = R(0), m1[2] = {R(0), R(0)}, m2[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int l = 0; l < Q; l++) {
        const R fl = f[l], c0 = R(cx(l)), c1 = R(cy(l));
        m0 += fl;
        m1[0] += fl * c0;
        m1[1] += fl * c1;
        m2[0] += fl * c0 * c0;
        m2[1] += fl * c0 * c1;
        m2[2] += fl * c1 * c1;
    }
    rho = sg * (R(1) + m0);
    j[0] = sg * m1[0];
    j[1] = sg * m1[1];
    Pi[0] = sg * (m2[0] + R(1.0 / 3.0));
    Pi[1] = sg * m2[1];
    Pi[2] = sg * (m2[2] + R(1.0 / 3.0));
}

// moments of f from h = f - w - F(t - dt)/2 and that history (A, B, C):
// rho = sqrt(g)(1 + sum h) + A/2, j = sqrt(g) sum h c + B/2,
// Pi = sqrt(g)(sum h c c + delta/3) + C/2 (sum F sqrt(g) = A, sum F c sqrt(g) = B, sum F c c sqrt(g) = C)
template <class R>
__device__ __forceinline__ void moments_h(const R h[Q], R sg, const R Fo[NF], R& rho, R j[2], R Pi[3])
{
    moments<R>(h, sg, rho, j, Pi);
    rho += R(0.5) * Fo[0];
    j[0] += R(0.5) * Fo[1];
    j[1] += R(0.5) * Fo[2];
    Pi[0] += R(0.5) * Fo[3];
    Pi[1] += R(0.5) * Fo[4];
    Pi[2] += R(0.5) * Fo[5];
}

// rule of a node on a non-periodic face (0: none), its inner node and face
__device__ __forceinline__ int classify(const Lat& L, int x, int y, int& axis, int& side, int& ix, int& iy)
{
    const int r[2] = {x, y};
    int in[2] = {x, y}, best = 0, rank = 0;
    const int prio[4] = {0, 3, 2, 1};
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int bc = s ? L.hi[a] : L.lo[a];
            if (bc == PER) continue;
            if (!(s ? r[a] == L.n[a] - 1 : r[a] == 0)) continue;
            in[a] = s ? r[a] - 1 : r[a] + 1;
            if (prio[bc] > rank) {
                rank = prio[bc];
                best = bc;
                axis = a;
                side = s;
            }
        }
    ix = in[0];
    iy = in[1];
    return best;
}

// the boundary rule of a face node (out of line: few nodes take it)
template <class R>
__device__ __noinline__ void face_pops(const Lat& L, const R* __restrict__ P, const R* __restrict__ Fc,
                                       const R* __restrict__ G, int x, int y, int bc, int axis, int side, int ix,
                                       int iy, R* f)
{
    const long long N = L.N, v = x + (long long)L.n[0] * y, vi = ix + (long long)L.n[0] * iy;
    R fi[Q];
    gather<R>(L, P, Fc, G, ix, iy, fi);
    Geo<R> gw, gin;
    load_geo(G, N, v, gw);
    load_geo(G, N, vi, gin);
    const R ratio = gin.sg * gw.isg;
    if (bc == OUTFLOW) {  // f_w = f_i ratio, so s_w = s_i ratio + w (ratio - 1)
#pragma unroll
        for (int l = 0; l < Q; l++) f[l] = fi[l] * ratio + R(wq(l)) * (ratio - R(1));
        return;
    }
    R rho, j[2], Pi[3];
    moments<R>(fi, gin.sg, rho, j, Pi);
    R uw[2] = {R(0), R(0)};
    const double* fv = L.face[axis * 2 + side];
    if (fv) {
        const int other = 1 - axis, nf = L.n[other], k = other == 0 ? x : y;
        uw[0] = R(fv[k]);
        uw[1] = R(fv[nf + k]);
    }
    const R jw[2] = {rho * uw[0], rho * uw[1]};
    R few[Q], fei[Q];
    feq_all<R>(gw, R(L.theta), rho, jw, few);
    feq_all<R>(gin, R(L.theta), rho, j, fei);
#pragma unroll
    for (int l = 0; l < Q; l++) f[l] = few[l] + (fi[l] - fei[l]) * ratio;
}

// what a node sees, in h-form: the pulled slots, or on a face node the
// boundary rule's s less F(t - dt)/2 of the node; Fo the node's history
template <class R>
__device__ __forceinline__ void node_state(const Lat& L, const R* __restrict__ P, const R* __restrict__ Fc,
                                           const R* __restrict__ G, int x, int y, R h[Q], R Fo[NF])
{
    const long long v = x + (long long)L.n[0] * y;
    load_fc(Fc, L.N, v, Fo);
    int axis = 0, side = 0, ix, iy;
    const int bc = classify(L, x, y, axis, side, ix, iy);
    if (bc == 0) {
        gather_h<R>(L, P, x, y, h);
    } else {
        R ff[Q];
        face_pops<R>(L, P, Fc, G, x, y, bc, axis, side, ix, iy, ff);
        const R isg = R(1) / G[v];
#pragma unroll
        for (int l = 0; l < Q; l++) h[l] = ff[l] - R(0.5) * forcing_l<R>(l, isg, Fo);
    }
}

// rho u at a site at most one step outside: periodic wrap or 2 j(face) - j(face - n), axis by axis
template <class R> __device__ __forceinline__ void jsite(const Lat& L, const R* __restrict__ jf, int x, int y, R out[2])
{
    int xs[2], ys[2];
    R wx[2], wy[2];
    int mx = 1, my = 1;
    auto axis_terms = [&](int a, int r, int* c, R* w, int& m) {
        int rr = r;
        if (wrap(L, a, rr)) {
            c[0] = rr;
            w[0] = R(1);
            m = 1;
        } else if (r < 0) {
            c[0] = 0;
            c[1] = 1;
            w[0] = R(2);
            w[1] = R(-1);
            m = 2;
        } else {
            c[0] = L.n[a] - 1;
            c[1] = L.n[a] - 2;
            w[0] = R(2);
            w[1] = R(-1);
            m = 2;
        }
    };
    axis_terms(0, x, xs, wx, mx);
    axis_terms(1, y, ys, wy, my);
    out[0] = out[1] = R(0);
    for (int b = 0; b < my; b++)
        for (int a = 0; a < mx; a++) {
            const long long v = xs[a] + (long long)L.n[0] * ys[b];
            const R w = wx[a] * wy[b];
            out[0] += w * jf[v];
            out[1] += w * jf[L.N + v];
        }
}

template <class R>
__global__ void __launch_bounds__(TB) k2_momentum(Lat L, const R* __restrict__ P, const R* __restrict__ Fc,
                                                  const R* __restrict__ G, R* __restrict__ jf)
{
    const long long v = blockIdx.x * (long long)TB + threadIdx.x;
    if (v >= L.N) return;
    const int x = (int)(v % L.n[0]), y = (int)(v / L.n[0]);
    R h[Q], Fo[NF], rho, j[2], Pi[3];
    node_state<R>(L, P, Fc, G, x, y, h, Fo);
    moments_h<R>(h, G[v], Fo, rho, j, Pi);
    jf[v] = j[0];
    jf[L.N + v] = j[1];
}

// the forcing coefficients of a node from its moments (rho, j, Pi), geometry
// and the rho u field; fe returns f^eq - w
template <class R>
__device__ __forceinline__ void forcing_coeffs(const Lat& L, const R* __restrict__ jf, int x, int y, const Geo<R>& g,
                                               R rho, const R j[2], const R Pi[3], R fe[Q], R out[NF])
{
    feq_all<R>(g, R(L.theta), rho, j, fe);
    // T = Pi^eq + (1 - 1/2tau) (Pi - Pi^eq)
    R Peq[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int l = 0; l < Q; l++) {
        const R c0 = R(cx(l)), c1 = R(cy(l)), fl = fe[l];
        Peq[0] += fl * c0 * c0;
        Peq[1] += fl * c0 * c1;
        Peq[2] += fl * c1 * c1;
    }
    Peq[0] = g.sg * (Peq[0] + R(1.0 / 3.0));
    Peq[1] = g.sg * Peq[1];
    Peq[2] = g.sg * (Peq[2] + R(1.0 / 3.0));
    R T[2][2];
    const R kv = R(L.kvisc);
    T[0][0] = Peq[0] + kv * (Pi[0] - Peq[0]);
    T[0][1] = T[1][0] = Peq[1] + kv * (Pi[1] - Peq[1]);
    T[1][1] = Peq[2] + kv * (Pi[2] - Peq[2]);
    // D[k][i] = 3 sum_l w_l c_l^k (rho u^i)(x + c_l); an interior node's
    // stencil needs no ghost (periodic wrap at most)
    R D[2][2] = {{R(0), R(0)}, {R(0), R(0)}};
    const bool inner = (x > 0 || L.lo[0] == PER) && (x < L.n[0] - 1 || L.hi[0] == PER) &&
                       (y > 0 || L.lo[1] == PER) && (y < L.n[1] - 1 || L.hi[1] == PER);
#pragma unroll
    for (int l = 1; l < Q; l++) {
        R jn[2];
        if (inner) {
            int xs = x + cx(l), ys = y + cy(l);
            wrap(L, 0, xs);
            wrap(L, 1, ys);
            const long long u = xs + (long long)L.n[0] * ys;
            jn[0] = jf[u];
            jn[1] = jf[L.N + u];
        } else {
            jsite<R>(L, jf, x + cx(l), y + cy(l), jn);
        }
        const R w = R(3.0 * wq(l));
#pragma unroll
        for (int i = 0; i < 2; i++) {
            D[0][i] += w * R(cx(l)) * jn[i];
            D[1][i] += w * R(cy(l)) * jn[i];
        }
    }
    auto gam = [&](int i, int a, int b) { return g.gam[i][s3(a, b)]; };
    auto gi = [&](int a, int b) { return g.gi[s3(a, b)]; };
    const R theta = R(L.theta);
    R A = R(0);
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = 0; k < 2; k++) A -= gam(i, i, k) * j[k] + gam(k, i, k) * j[i];
    R B[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        R b = R(L.fext[i]);
#pragma unroll
        for (int jj = 0; jj < 2; jj++)
#pragma unroll
            for (int k = 0; k < 2; k++)
                b -= gam(k, jj, k) * T[i][jj] + gam(i, jj, k) * T[jj][k] + gam(jj, jj, k) * T[k][i];
        B[i] = b;
    }
    R bard[2][2], cov[2][2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const R trace = gam(0, k, 0) + gam(1, k, 1);
#pragma unroll
        for (int i = 0; i < 2; i++) {
            bard[k][i] = D[k][i] - trace * j[i];
            cov[k][i] = D[k][i] + gam(i, k, 0) * j[0] + gam(i, k, 1) * j[1];
        }
    }
    const R divbar = bard[0][0] + bard[1][1], divcov = cov[0][0] + cov[1][1];
    R C[3];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int jj = i; jj < 2; jj++) {
            R s = R(1.0 / 3.0) * (bard[jj][i] + bard[i][jj] + (i == jj ? divbar : R(0)));
#pragma unroll
            for (int k = 0; k < 2; k++) s -= theta * (cov[k][i] * gi(jj, k) + cov[k][jj] * gi(i, k));
            s -= theta * divcov * gi(i, jj);
            C[s3(i, jj)] = s;
        }
    out[0] = A;
    out[1] = B[0];
    out[2] = B[1];
    out[3] = C[0];
    out[4] = C[1];
    out[5] = C[2];
}

// the forcing coefficients of a node from its moments, geometry and the
// lattice gradient D[k][i] = d_k (rho u^i) (Eqs. forcing-A/B/C), and the
// first two Hermite coefficients of f^eq - w (a0e, a2e; the first is j).
// The equilibrium flux is Pi^eq = sum_l f^eq_l c c sqrt(g) = rho theta g^ij
// + j^i j^j / rho: the second moment of the second-order Hermite expansion
// on D2Q9 (sum w c c = delta / 3, sum w c c c c = (delta delta + 2 perms) / 9)
template <class R>
__device__ __forceinline__ void forcing_from_gradient(const Lat& L, const Geo<R>& g, R rho, const R j[2],
                                                      const R Pi[3], const R D[2][2], R& a0e, R a2e[3], R out[NF])
{
    const R ir = R(1) / rho, theta = R(L.theta);
    R Peq[3];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = i; k < 2; k++) {
            const R jj = j[i] * j[k] * ir;
            Peq[s3(i, k)] = rho * theta * g.gi[s3(i, k)] + jj;
            a2e[s3(i, k)] = rho * (theta * g.gi[s3(i, k)] - (i == k ? R(1.0 / 3.0) : R(0))) + jj;
        }
    a0e = rho - g.sg;
    R T[2][2];
    const R kv = R(L.kvisc);
    T[0][0] = Peq[0] + kv * (Pi[0] - Peq[0]);
    T[0][1] = T[1][0] = Peq[1] + kv * (Pi[1] - Peq[1]);
    T[1][1] = Peq[2] + kv * (Pi[2] - Peq[2]);
    auto gam = [&](int i, int a, int b) { return g.gam[i][s3(a, b)]; };
    auto gi = [&](int a, int b) { return g.gi[s3(a, b)]; };
    R A = R(0);
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = 0; k < 2; k++) A -= gam(i, i, k) * j[k] + gam(k, i, k) * j[i];
    R B[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        R b = R(L.fext[i]);
#pragma unroll
        for (int jj = 0; jj < 2; jj++)
#pragma unroll
            for (int k = 0; k < 2; k++)
                b -= gam(k, jj, k) * T[i][jj] + gam(i, jj, k) * T[jj][k] + gam(jj, jj, k) * T[k][i];
        B[i] = b;
    }
    R bard[2][2], cov[2][2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const R trace = gam(0, k, 0) + gam(1, k, 1);
#pragma unroll
        for (int i = 0; i < 2; i++) {
            bard[k][i] = D[k][i] - trace * j[i];
            cov[k][i] = D[k][i] + gam(i, k, 0) * j[0] + gam(i, k, 1) * j[1];
        }
    }
    const R divbar = bard[0][0] + bard[1][1], divcov = cov[0][0] + cov[1][1];
    R C[3];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int jj = i; jj < 2; jj++) {
            R sc = R(1.0 / 3.0) * (bard[jj][i] + bard[i][jj] + (i == jj ? divbar : R(0)));
#pragma unroll
            for (int k = 0; k < 2; k++) sc -= theta * (cov[k][i] * gi(jj, k) + cov[k][jj] * gi(i, k));
            sc -= theta * divcov * gi(i, jj);
            C[s3(i, jj)] = sc;
        }
    out[0] = A;
    out[1] = B[0];
    out[2] = B[1];
    out[3] = C[0];
    out[4] = C[1];
    out[5] = C[2];
}

// ---------------------------------------------------------------------------
// The step in one pass, marching along y.  A block of SW threads owns a strip
// of SW - 2 columns (thread t at column x0 - 1 + t; threads 0 and SW - 1 only
// supply rho u of the two columns beside the strip) and a band of rows, which
// it walks upwards.  For row c it forms the state and rho u of row c + 1 (the
// pulled slots, the history, sqrt(g)) into a ring of four rho u rows in shared
// memory, then steps row c with the gradient stencil read from the ring, the
// state of row c kept in registers from the iteration before.  Every slot is
// read once; rho u of the columns beside a strip and of the rows beside a
// band is formed twice (by both neighbours).  A stencil site past a
// non-periodic face takes the linear ghost 2 j(face) - j(face - n), axis by
// axis.
// ---------------------------------------------------------------------------

// a row index past an end: wrapped on a periodic axis, else false
__device__ __forceinline__ bool wrap_row(const Lat& L, int& r)
{
    if (r >= 0 && r < L.n[1]) return true;
    if (L.lo[1] != PER) return false;
    r += r < 0 ? L.n[1] : -L.n[1];
    return true;
}

// h, the history and rho u, Pi of node (x, y).  `fast`: an interior node
// whose pull sources lie inside the lattice without wrapping
template <class R>
__device__ __forceinline__ void march_state(const Lat& L, const R* __restrict__ P, const R* __restrict__ Fc,
                                            const R* __restrict__ G, int x, int y, bool fast, R h[Q], R Fo[NF],
                                            R& rho, R j[2], R Pi[3])
{
    const long long N = L.N, v = x + (long long)L.n[0] * y;
    if (fast) {
        load_fc(Fc, N, v, Fo);
#pragma unroll
        for (int l = 0; l < Q; l++) h[l] = P[l * N + v - cx(l) - (long long)L.n[0] * cy(l)];
    } else {
        node_state<R>(L, P, Fc, G, x, y, h, Fo);
    }
    moments_h<R>(h, G[v], Fo, rho, j, Pi);
}

// rho u at stencil site (t + dx, row slot of c + dy) of the ring, ghosts
// past non-periodic faces extrapolated axis by axis; gx is thread t's column
template <class R, int SW>
__device__ __forceinline__ void ring_site(const Lat& L, const R (*ring)[2][SW], int t, int gx, int c, int m, int dx,
                                          int dy, R out[2])
{
    // two terms per axis; the second has weight 0 unless the site is a ghost
    int xa = t + dx, xb = t + dx, ma = m + dy, mb = m + dy;
    R wxa = R(1), wxb = R(0), wya = R(1), wyb = R(0);
    const int sx = gx + dx, sy = c + dy;
    if (sx < 0 && L.lo[0] != PER) { xa = t + dx + 1; xb = t + dx + 2; wxa = R(2); wxb = R(-1); }
    else if (sx >= L.n[0] && L.hi[0] != PER) { xa = t + dx - 1; xb = t + dx - 2; wxa = R(2); wxb = R(-1); }
    if (sy < 0 && L.lo[1] != PER) { ma = m + dy + 1; mb = m + dy + 2; wya = R(2); wyb = R(-1); }
    else if (sy >= L.n[1] && L.hi[1] != PER) { ma = m + dy - 1; mb = m + dy - 2; wya = R(2); wyb = R(-1); }
#pragma unroll
    for (int i = 0; i < 2; i++)
        out[i] = wya * (wxa * ring[ma & 3][i][xa] + wxb * ring[ma & 3][i][xb]) +
                 wyb * (wxa * ring[mb & 3][i][xa] + wxb * ring[mb & 3][i][xb]);
}

// blocks per SM the register budget is set for: 16 warps (FP32), 8 (FP64)
template <class R, int SW> constexpr int march_min_blocks() { return (sizeof(R) == 8 ? 256 : 512) / SW; }

template <class R, int SW>
__global__ void __launch_bounds__(SW, march_min_blocks<R, SW>())
    k2_step_march(Lat L, const R* __restrict__ P, R* __restrict__ Pout, const R* __restrict__ Fc,
                  R* __restrict__ Fout, const R* __restrict__ G, int nstrip, int H, int nitems)
{
    __shared__ R ring[4][2][SW];
    const int t = threadIdx.x, n0 = L.n[0], n1 = L.n[1];
    const long long N = L.N;
    const bool xper = L.lo[0] == PER;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int s = item % nstrip, band = item / nstrip;
        const int x0 = s * (SW - 2), ya = band * H, yb = min(n1, ya + H);
        const int gx = x0 - 1 + t;
        // the column whose rho u this thread forms (wrapped), -1 for none
        int mxc = gx;
        if (gx < 0) mxc = xper ? gx + n0 : -1;
        else if (gx >= n0) mxc = (gx == n0 && xper) ? 0 : -1;
        const bool stepper = t >= 1 && t <= SW - 2 && gx < n0;
        // every column of the strip and its pull sources inside, no face column
        const bool fastx = x0 >= 2 && x0 + SW <= n0;
        R h[Q], Fo[NF], rho = R(1), j[2] = {R(0), R(0)}, Pi[3] = {R(0), R(0), R(0)};
        // ring slot of row ya - 1 + m is m & 3: rows ya - 1 and ya first
        {
            int r = ya - 1;
            if (mxc >= 0 && wrap_row(L, r)) {
                R hh[Q], FF[NF], rr, jj[2], PP[3];
                march_state<R>(L, P, Fc, G, mxc, r, fastx && r >= 1 && r <= n1 - 2, hh, FF, rr, jj, PP);
                ring[0][0][t] = jj[0];
                ring[0][1][t] = jj[1];
            }
            if (mxc >= 0) {
                march_state<R>(L, P, Fc, G, mxc, ya, fastx && ya >= 1 && ya <= n1 - 2, h, Fo, rho, j, Pi);
                ring[1][0][t] = j[0];
                ring[1][1][t] = j[1];
            }
        }
        for (int c = ya; c < yb; c++) {
            const int m = c - ya + 1;
            // row c + 1 into the ring (its state kept for the next iteration)
            R hn[Q], Fon[NF], rhon = R(1), jn[2] = {R(0), R(0)}, Pin[3] = {R(0), R(0), R(0)};
            int r = c + 1;
            if (mxc >= 0 && wrap_row(L, r)) {
                march_state<R>(L, P, Fc, G, mxc, r, fastx && r >= 1 && r <= n1 - 2, hn, Fon, rhon, jn, Pin);
                ring[(m + 1) & 3][0][t] = jn[0];
                ring[(m + 1) & 3][1][t] = jn[1];
            }
            __syncthreads();
            if (stepper) {
                const long long v = gx + (long long)n0 * c;
                Geo<R> g;
                load_geo(G, N, v, g);
                R D[2][2] = {{R(0), R(0)}, {R(0), R(0)}};
                if (fastx && c >= 1 && c <= n1 - 2) {
#pragma unroll
                    for (int l = 1; l < Q; l++) {
                        const R w = R(3.0 * wq(l));
                        const int sl = (m + cy(l)) & 3;
#pragma unroll
                        for (int i = 0; i < 2; i++) {
                            const R jl = ring[sl][i][t + cx(l)];
                            D[0][i] += w * R(cx(l)) * jl;
                            D[1][i] += w * R(cy(l)) * jl;
                        }
                    }
                } else {
#pragma unroll
                    for (int l = 1; l < Q; l++) {
                        R jl[2];
                        ring_site<R, SW>(L, ring, t, gx, c, m, cx(l), cy(l), jl);
                        const R w = R(3.0 * wq(l));
#pragma unroll
                        for (int i = 0; i < 2; i++) {
                            D[0][i] += w * R(cx(l)) * jl[i];
                            D[1][i] += w * R(cy(l)) * jl[i];
                        }
                    }
                }
                R Fn[NF], a0e, a2e[3];
                forcing_from_gradient<R>(L, g, rho, j, Pi, D, a0e, a2e, Fn);
                // f* - w = (1 - omega) h + omega (f^eq - w) + F(t) - omega F(t - dt)/2 (s = h
                // + F(t - dt)/2): one Hermite recomposition of the combined coefficients
                const R om = R(L.omega);
                R K[NF];
#pragma unroll
                for (int k = 0; k < NF; k++) K[k] = Fn[k] - R(0.5) * om * Fo[k];
                const R c0 = om * a0e + K[0];
                const R c1[2] = {om * j[0] + K[1], om * j[1] + K[2]};
                const R c2[3] = {om * a2e[0] + K[3] - K[0] * R(1.0 / 3.0), om * a2e[1] + K[4],
                                 om * a2e[2] + K[5] - K[0] * R(1.0 / 3.0)};
#pragma unroll
                for (int l = 0; l < Q; l++) Pout[l * N + v] = (R(1) - om) * h[l] + hermite<R>(l, g.isg, c0, c1, c2);
#pragma unroll
                for (int k = 0; k < NF; k++) Fout[k * N + v] = Fn[k];
            }
#pragma unroll
            for (int l = 0; l < Q; l++) h[l] = hn[l];
#pragma unroll
            for (int k = 0; k < NF; k++) Fo[k] = Fon[k];
            rho = rhon;
            j[0] = jn[0];
            j[1] = jn[1];
            Pi[0] = Pin[0];
            Pi[1] = Pin[1];
            Pi[2] = Pin[2];
        }
        __syncthreads();  // the ring is free for the next item
    }
}

// initialisation: slots so that the gather returns f^eq with no forcing yet
template <class R>
__global__ void __launch_bounds__(TB) k2_init_eq(Lat L, const double* __restrict__ rho0, const double* __restrict__ u0,
                                                 R* __restrict__ P, R* __restrict__ Fc, const R* __restrict__ G)
{
    const long long v = blockIdx.x * (long long)TB + threadIdx.x;
    if (v >= L.N) return;
    const long long N = L.N;
    const int x = (int)(v % L.n[0]), y = (int)(v / L.n[0]);
    Geo<R> g;
    load_geo(G, N, v, g);
    const R rho = rho0 ? R(rho0[v]) : R(1);
    const R j[2] = {u0 ? rho * R(u0[v]) : R(0), u0 ? rho * R(u0[N + v]) : R(0)};
    R fe[Q];
    feq_all<R>(g, R(L.theta), rho, j, fe);
#pragma unroll
    for (int l = 0; l < Q; l++) {
        int xs = x - cx(l), ys = y - cy(l);
        if (!wrap(L, 0, xs) || !wrap(L, 1, ys)) continue;
        P[l * N + xs + (long long)L.n[0] * ys] = fe[l];
    }
#pragma unroll
    for (int k = 0; k < NF; k++) Fc[k * N + v] = R(0);
}

// F(0) of the initial state into the history (F(-dt) := F(0))
template <class R>
__global__ void __launch_bounds__(TB) k2_init_force(Lat L, const R* __restrict__ P, const R* __restrict__ Fc0,
                                                    R* __restrict__ Fc, const R* __restrict__ G,
                                                    const R* __restrict__ jf)
{
    const long long v = blockIdx.x * (long long)TB + threadIdx.x;
    if (v >= L.N) return;
    const int x = (int)(v % L.n[0]), y = (int)(v / L.n[0]);
    R h[Q], Fo[NF];
    node_state<R>(L, P, Fc0, G, x, y, h, Fo);
    Geo<R> g;
    load_geo(G, L.N, v, g);
    R rho, j[2], Pi[3], fe[Q], Fn[NF];
    moments_h<R>(h, g.sg, Fo, rho, j, Pi);
    forcing_coeffs<R>(L, jf, x, y, g, rho, j, Pi, fe, Fn);
#pragma unroll
    for (int k = 0; k < NF; k++) Fc[k * L.N + v] = Fn[k];
}

// the slots the node pulls lose F/2 of the node's new history, so that the
// gather (slot + F/2) still returns the initial populations
template <class R>
__global__ void __launch_bounds__(TB) k2_half_shift(Lat L, R* __restrict__ P, const R* __restrict__ Fc,
                                                    const R* __restrict__ G)
{
    const long long v = blockIdx.x * (long long)TB + threadIdx.x;
    if (v >= L.N) return;
    const long long N = L.N;
    const int x = (int)(v % L.n[0]), y = (int)(v / L.n[0]);
    R fc[NF];
    load_fc(Fc, N, v, fc);
    const R isg = R(1) / G[v];
#pragma unroll
    for (int l = 0; l < Q; l++) {
        int xs = x - cx(l), ys = y - cy(l);
        if (!wrap(L, 0, xs) || !wrap(L, 1, ys)) continue;
        P[l * N + xs + (long long)L.n[0] * ys] -= R(0.5) * forcing_l<R>(l, isg, fc);
    }
}

// g^ij, sqrt(g), Gamma^i_jk from g_ij and d_k g_ij (FP64 inversion, App. A)
template <class R>
__global__ void __launch_bounds__(TB) k2_metric(long long N, const double* __restrict__ g3, const double* __restrict__ dg6,
                                                R* __restrict__ G, int* bad)
{
    const long long v = blockIdx.x * (long long)TB + threadIdx.x;
    if (v >= N) return;
    const double g00 = g3[v], g01 = g3[N + v], g11 = g3[2 * N + v];
    const double det = g00 * g11 - g01 * g01;
    if (!(det > 0.0)) {
        atomicOr(bad, 1);
        return;
    }
    const double id = 1.0 / det;
    const double gi[2][2] = {{g11 * id, -g01 * id}, {-g01 * id, g00 * id}};
    double dg[2][2][2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        dg[k][0][0] = dg6[(k * 3 + 0) * N + v];
        dg[k][0][1] = dg[k][1][0] = dg6[(k * 3 + 1) * N + v];
        dg[k][1][1] = dg6[(k * 3 + 2) * N + v];
    }
    G[v] = R(sqrt(det));
    G[N + v] = R(gi[0][0]);
    G[2 * N + v] = R(gi[0][1]);
    G[3 * N + v] = R(gi[1][1]);
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int p = 0; p < 3; p++) {
            const int a = p == 2 ? 1 : 0, b = p == 0 ? 0 : 1;
            double s = 0.0;
#pragma unroll
            for (int l = 0; l < 2; l++) s += gi[i][l] * (dg[a][b][l] + dg[b][a][l] - dg[l][a][b]);
            G[(4 + i * 3 + p) * N + v] = R(0.5 * s);
        }
}

// node-wise chart change: D = Jn^-1 Jo; rho kept, j -> D j, Pi -> D Pi D^T,
// recomposed with the new sqrt(g); the history A, D B, D C D^T; the new
// populations scattered to the slots they are pulled from
template <class R>
__global__ void __launch_bounds__(TB) k2_transform(Lat L, const R* __restrict__ P, R* __restrict__ Pout,
                                                   const R* __restrict__ Fc, R* __restrict__ Fout,
                                                   const R* __restrict__ Gold, const R* __restrict__ Gnew,
                                                   const double* __restrict__ Jo4, const double* __restrict__ Jn4)
{
    const long long v = blockIdx.x * (long long)TB + threadIdx.x;
    if (v >= L.N) return;
    const long long N = L.N;
    const int x = (int)(v % L.n[0]), y = (int)(v / L.n[0]);
    R h[Q], rho, j[2], Pi[3], fc[NF];
    node_state<R>(L, P, Fc, Gold, x, y, h, fc);
    moments_h<R>(h, Gold[v], fc, rho, j, Pi);
    const double a = Jn4[v], b = Jn4[N + v], c = Jn4[2 * N + v], d = Jn4[3 * N + v], id = 1.0 / (a * d - b * c);
    const double ni[2][2] = {{d * id, -b * id}, {-c * id, a * id}};
    const double o[2][2] = {{Jo4[v], Jo4[N + v]}, {Jo4[2 * N + v], Jo4[3 * N + v]}};
    R D[2][2];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = 0; k < 2; k++) D[i][k] = R(ni[i][0] * o[0][k] + ni[i][1] * o[1][k]);
    auto vec = [&](const R in[2], R out[2]) {
        out[0] = D[0][0] * in[0] + D[0][1] * in[1];
        out[1] = D[1][0] * in[0] + D[1][1] * in[1];
    };
    auto ten = [&](const R in[3], R out[3]) {
        const R M[2][2] = {{in[0], in[1]}, {in[1], in[2]}};
        R t[2][2];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int m = 0; m < 2; m++) t[i][m] = D[i][0] * M[0][m] + D[i][1] * M[1][m];
        out[0] = t[0][0] * D[0][0] + t[0][1] * D[0][1];
        out[1] = t[0][0] * D[1][0] + t[0][1] * D[1][1];
        out[2] = t[1][0] * D[1][0] + t[1][1] * D[1][1];
    };
    R j2[2], P2[3], Fn[NF];
    vec(j, j2);
    ten(Pi, P2);
    P2[0] -= rho * R(1.0 / 3.0);
    P2[2] -= rho * R(1.0 / 3.0);
    Fn[0] = fc[0];
    {
        const R Bo[2] = {fc[1], fc[2]}, Co[3] = {fc[3], fc[4], fc[5]};
        R Bn[2], Cn[3];
        vec(Bo, Bn);
        ten(Co, Cn);
        Fn[1] = Bn[0];
        Fn[2] = Bn[1];
        Fn[3] = Cn[0];
        Fn[4] = Cn[1];
        Fn[5] = Cn[2];
    }
    const R isgn = R(1) / Gnew[v];
#pragma unroll
    for (int k = 0; k < NF; k++) Fout[k * N + v] = Fn[k];
#pragma unroll
    for (int l = 0; l < Q; l++) {
        int xs = x - cx(l), ys = y - cy(l);
        if (!wrap(L, 0, xs) || !wrap(L, 1, ys)) continue;
        Pout[l * N + xs + (long long)L.n[0] * ys] =
            hermite<R>(l, isgn, rho - Gnew[v], j2, P2) - R(0.5) * forcing_l<R>(l, isgn, Fn);
    }
}

template <class R>
__global__ void __launch_bounds__(TB) k2_readout(Lat L, const R* __restrict__ P, const R* __restrict__ Fc,
                                                 const R* __restrict__ G, const double* __restrict__ J4,
                                                 double* __restrict__ rho_out, double* __restrict__ u_out,
                                                 int cartesian)
{
    const long long v = blockIdx.x * (long long)TB + threadIdx.x;
    if (v >= L.N) return;
    const long long N = L.N;
    const int x = (int)(v % L.n[0]), y = (int)(v / L.n[0]);
    R h[Q], Fo[NF], rho, j[2], Pi[3];
    node_state<R>(L, P, Fc, G, x, y, h, Fo);
    moments_h<R>(h, G[v], Fo, rho, j, Pi);
    const double u0 = double(j[0]) / double(rho), u1 = double(j[1]) / double(rho);
    rho_out[v] = double(rho);
    if (cartesian) {
        u_out[v] = J4[v] * u0 + J4[N + v] * u1;
        u_out[N + v] = J4[2 * N + v] * u0 + J4[3 * N + v] * u1;
    } else {
        u_out[v] = u0;
        u_out[N + v] = u1;
    }
}

template <int K> __device__ __forceinline__ void block_add(double (&val)[K], double* acc)
{
    __shared__ double part[K][TB / 32];
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val[k] += __shfl_down_sync(0xffffffffu, val[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) part[k][wid] = val[k];
    __syncthreads();
    if (wid == 0)
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = lane < TB / 32 ? part[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) atomicAdd(acc + k, s);
        }
}

template <class R>
__global__ void __launch_bounds__(TB) k2_mass(Lat L, const R* __restrict__ P, const R* __restrict__ Fc,
                                              const R* __restrict__ G, double* acc)
{
    const long long v = blockIdx.x * (long long)TB + threadIdx.x;
    double val[1] = {0.0};
    if (v < L.N) {
        const int x = (int)(v % L.n[0]), y = (int)(v / L.n[0]);
        R h[Q], Fo[NF], rho, j[2], Pi[3];
        node_state<R>(L, P, Fc, G, x, y, h, Fo);
        moments_h<R>(h, G[v], Fo, rho, j, Pi);
        val[0] = double(G[v]) * double(rho);
    }
    block_add<1>(val, acc);
}

// F^a = s sum_{face nodes} J^a_i T^{i axis} sqrt(g)
template <class R>
__global__ void __launch_bounds__(TB) k2_wall_force(Lat L, const R* __restrict__ P, const R* __restrict__ Fc,
                                                    const R* __restrict__ G, const double* __restrict__ J4, int axis,
                                                    int side, double* acc)
{
    const int other = 1 - axis;
    const long long t = blockIdx.x * (long long)TB + threadIdx.x;
    double val[2] = {0.0, 0.0};
    if (t < L.n[other]) {
        int r[2];
        r[axis] = side ? L.n[axis] - 1 : 0;
        r[other] = (int)t;
        const long long N = L.N, v = r[0] + (long long)L.n[0] * r[1];
        R h[Q], Fo[NF], rho, j[2], Pi[3], fe[Q];
        node_state<R>(L, P, Fc, G, r[0], r[1], h, Fo);
        Geo<R> g;
        load_geo(G, N, v, g);
        moments_h<R>(h, g.sg, Fo, rho, j, Pi);
        feq_all<R>(g, R(L.theta), rho, j, fe);
        R Peq[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int l = 0; l < Q; l++) {
            const R c0 = R(cx(l)), c1 = R(cy(l)), fl = fe[l];
            Peq[0] += fl * c0 * c0;
            Peq[1] += fl * c0 * c1;
            Peq[2] += fl * c1 * c1;
        }
        Peq[0] = g.sg * (Peq[0] + R(1.0 / 3.0));
        Peq[1] = g.sg * Peq[1];
        Peq[2] = g.sg * (Peq[2] + R(1.0 / 3.0));
        const R kv = R(L.kvisc);
        const R T[2][2] = {{Peq[0] + kv * (Pi[0] - Peq[0]), Peq[1] + kv * (Pi[1] - Peq[1])},
                           {Peq[1] + kv * (Pi[1] - Peq[1]), Peq[2] + kv * (Pi[2] - Peq[2])}};
        const double s = side ? 1.0 : -1.0;
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int i = 0; i < 2; i++) val[a] += s * J4[(a * 2 + i) * N + v] * double(T[i][axis]) * double(g.sg);
    }
    block_add<2>(val, acc);
}

}  // namespace cslbm2d

using namespace cslbm2d;

struct cslbm2d_ctx {
    cslbm2d_params p;
    long long N;
    cudaStream_t stream;
    size_t r;         // bytes per value (4 or 8)
    void* P[2];       // [9][N] slots
    void* F[2];       // [6][N] forcing coefficients
    void* G[2];       // [10][N] geometry
    void* jf;         // [2][N] rho u
    double* J;        // [4][N]
    double* face[4];  // [2][n other] per face
    double* stage;    // host-input staging, 10 N doubles
    double* scratch;  // 64 doubles
    int pc, gc, has_state, has_metric;
    int march_blocks;  // resident blocks of the marching step (0: not yet known)
};

namespace {

cslbm_status fail2(cslbm_status s, const std::string& m) { return cslbm_record_error(s, m.c_str()); }

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

bool params_ok(const cslbm2d_params* p, std::string& why)
{
    for (int a = 0; a < 2; a++) {
        if (p->n[a] < 1) return why = "n must be positive", false;
        if ((p->bc_lo[a] == PER) != (p->bc_hi[a] == PER)) return why = "an axis is periodic on both sides or neither", false;
        if (p->bc_lo[a] < 0 || p->bc_lo[a] > 3 || p->bc_hi[a] < 0 || p->bc_hi[a] > 3) return why = "unknown rule", false;
        if (p->bc_lo[a] != PER && p->n[a] < 3) return why = "a non-periodic axis needs 3 nodes", false;
    }
    if (!(p->tau > 0.5)) return why = "tau must exceed 1/2", false;
    if (p->storage != CSLBM_FP32 && p->storage != CSLBM_FP64) return why = "2-D storage is FP32 or FP64", false;
    return true;
}

size_t layout(const cslbm2d_params* p, size_t off[12])
{
    const size_t N = (size_t)p->n[0] * p->n[1], r = p->storage == CSLBM_FP64 ? 8 : 4;
    const size_t sz[12] = {9 * N * r, 9 * N * r, 6 * N * r, 6 * N * r, 10 * N * r, 10 * N * r, 2 * N * r, 4 * N * 8,
                           2 * (size_t)(p->n[0] + p->n[1]) * 2 * 8, 10 * N * 8, 64 * 8, 0};
    size_t o = 0;
    for (int k = 0; k < 11; k++) {
        off[k] = o;
        o += align256(sz[k]);
    }
    return o;
}

Lat lat_of(const cslbm2d_ctx* c)
{
    Lat L;
    for (int a = 0; a < 2; a++) {
        L.n[a] = c->p.n[a];
        L.lo[a] = c->p.bc_lo[a];
        L.hi[a] = c->p.bc_hi[a];
        L.fext[a] = c->p.fext[a];
    }
    L.N = c->N;
    L.omega = 1.0 / c->p.tau;
    L.kvisc = 1.0 - 0.5 / c->p.tau;
    L.theta = c->p.theta > 0 ? c->p.theta : 1.0 / 3.0;
    for (int k = 0; k < 4; k++) L.face[k] = c->face[k];
    return L;
}

unsigned nb(long long n) { return (unsigned)((n + TB - 1) / TB); }

// a device copy of an FP64 input (staged through the workspace when on the host)
cslbm_status in64(cslbm2d_ctx* c, const double* src, size_t count, int on_device, const double** out)
{
    if (on_device) {
        *out = src;
        return CSLBM_OK;
    }
    if (count > 10 * (size_t)c->N) return fail2(CSLBM_EINVAL, "input larger than the staging area");
    if (cudaMemcpyAsync(c->stage, src, count * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return fail2(CSLBM_ECUDA, "copy to the device failed");
    *out = c->stage;
    return CSLBM_OK;
}

cslbm_status launched(cslbm2d_ctx* c, const char* what, bool sync = false)
{
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && sync) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail2(CSLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return CSLBM_OK;
}

template <class R> cslbm_status metric(cslbm2d_ctx* c, const double* g3, const double* dg6, int dst)
{
    int* bad = (int*)(c->scratch + 32);
    cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    k2_metric<R><<<nb(c->N), TB, 0, c->stream>>>(c->N, g3, dg6, (R*)c->G[dst], bad);
    int h = 0;
    cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (cslbm_status s = launched(c, "metric kernel", true)) return s;
    if (h) return fail2(CSLBM_EINVAL, "metric not positive definite");
    return CSLBM_OK;
}

// Work items of the marching step: strips of SW - 2 columns times bands of H
// rows, H chosen so that the rounds of resident blocks times the rows a block
// forms (H + 2) are fewest
constexpr int SW = 64;

template <class R> void step_once(cslbm2d_ctx* c)
{
    const Lat L = lat_of(c);
    const int i = c->pc, o = 1 - c->pc;
    if (!c->march_blocks) {
        int dev = 0, nsm = 1, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k2_step_march<R, SW>, SW, 0);
        c->march_blocks = (per > 0 ? per : 1) * nsm;
    }
    const int nstrip = (L.n[0] + SW - 3) / (SW - 2), n1 = L.n[1];
    long long best = -1;
    int H = n1;
    for (int nb = 1; nb <= n1; nb++) {
        const int h = (n1 + nb - 1) / nb, bands = (n1 + h - 1) / h;
        const long long items = (long long)nstrip * bands;
        const long long cost = (items + c->march_blocks - 1) / c->march_blocks * (h + 2);
        if (best < 0 || cost < best) {
            best = cost;
            H = h;
        }
    }
    const int nitems = nstrip * ((n1 + H - 1) / H);
    const int grid = nitems < c->march_blocks ? nitems : c->march_blocks;
    k2_step_march<R, SW><<<grid, SW, 0, c->stream>>>(L, (const R*)c->P[i], (R*)c->P[o], (const R*)c->F[i],
                                                     (R*)c->F[o], (const R*)c->G[c->gc], nstrip, H, nitems);
    c->pc = o;
}

template <class R> void init(cslbm2d_ctx* c, const double* rho, const double* u)
{
    const Lat L = lat_of(c);
    const int i = c->pc, o = 1 - c->pc;
    const R* G = (const R*)c->G[c->gc];
    k2_init_eq<R><<<nb(c->N), TB, 0, c->stream>>>(L, rho, u, (R*)c->P[i], (R*)c->F[o], G);
    // rho u and F(0) of the boundary-filled initial state (no forcing yet: F[o] is zero)
    k2_momentum<R><<<nb(c->N), TB, 0, c->stream>>>(L, (const R*)c->P[i], (const R*)c->F[o], G, (R*)c->jf);
    k2_init_force<R><<<nb(c->N), TB, 0, c->stream>>>(L, (const R*)c->P[i], (const R*)c->F[o], (R*)c->F[i], G,
                                                     (const R*)c->jf);
    k2_half_shift<R><<<nb(c->N), TB, 0, c->stream>>>(L, (R*)c->P[i], (const R*)c->F[i], G);
}

template <class R> cslbm_status transform(cslbm2d_ctx* c, const double* Jn)
{
    const Lat L = lat_of(c);
    const int i = c->pc, o = 1 - c->pc;
    k2_transform<R><<<nb(c->N), TB, 0, c->stream>>>(L, (const R*)c->P[i], (R*)c->P[o], (const R*)c->F[i], (R*)c->F[o],
                                                    (const R*)c->G[c->gc], (const R*)c->G[1 - c->gc], c->J, Jn);
    return launched(c, "transform kernel");
}

}  // namespace

#define DISPATCH(c, call) ((c)->r == 8 ? call<double> : call<float>)

extern "C" {

cslbm_status cslbm2d_workspace_bytes(const cslbm2d_params* p, size_t* bytes)
{
    std::string why;
    if (!p || !bytes) return fail2(CSLBM_EINVAL, "null argument");
    if (!params_ok(p, why)) return fail2(CSLBM_EINVAL, why);
    size_t off[12];
    *bytes = layout(p, off);
    return CSLBM_OK;
}

cslbm_status cslbm2d_create(const cslbm2d_params* p, void* ws, size_t bytes, void* stream, cslbm2d_ctx** out)
{
    size_t need = 0;
    if (cslbm_status s = cslbm2d_workspace_bytes(p, &need)) return s;
    if (!ws || !out) return fail2(CSLBM_EINVAL, "null argument");
    if (bytes < need) return fail2(CSLBM_ENOMEM, "workspace smaller than required");
    if ((uintptr_t)ws & 255) return fail2(CSLBM_EINVAL, "workspace must be 256-byte aligned");
    cslbm2d_ctx* c = new cslbm2d_ctx();
    c->p = *p;
    c->N = (long long)p->n[0] * p->n[1];
    c->stream = (cudaStream_t)stream;
    c->r = p->storage == CSLBM_FP64 ? 8 : 4;
    size_t off[12];
    layout(p, off);
    char* b = (char*)ws;
    c->P[0] = b + off[0];
    c->P[1] = b + off[1];
    c->F[0] = b + off[2];
    c->F[1] = b + off[3];
    c->G[0] = b + off[4];
    c->G[1] = b + off[5];
    c->jf = b + off[6];
    c->J = (double*)(b + off[7]);
    for (int a = 0; a < 2; a++)
        for (int s = 0; s < 2; s++) c->face[a * 2 + s] = nullptr;
    c->stage = (double*)(b + off[9]);
    c->scratch = (double*)(b + off[10]);
    if (cudaMemsetAsync(ws, 0, need, c->stream) != cudaSuccess) {
        delete c;
        return fail2(CSLBM_ECUDA, "memset failed");
    }
    // identity Jacobian until set
    double* Jh = new double[4 * c->N];
    for (long long v = 0; v < c->N; v++) {
        Jh[v] = 1.0;
        Jh[c->N + v] = 0.0;
        Jh[2 * c->N + v] = 0.0;
        Jh[3 * c->N + v] = 1.0;
    }
    cudaError_t e = cudaMemcpyAsync(c->J, Jh, 4 * c->N * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    delete[] Jh;
    if (e != cudaSuccess) {
        delete c;
        return fail2(CSLBM_ECUDA, "initial copy failed");
    }
    *out = c;
    return CSLBM_OK;
}

cslbm_status cslbm2d_destroy(cslbm2d_ctx* c)
{
    delete c;
    return CSLBM_OK;
}

cslbm_status cslbm2d_set_metric(cslbm2d_ctx* c, const double* g3, const double* dg6, int on_device)
{
    if (!c || !g3 || !dg6) return fail2(CSLBM_EINVAL, "null argument");
    const double *dg, *gg;
    if (on_device) {
        gg = g3;
        dg = dg6;
    } else {
        if (cudaMemcpyAsync(c->stage, g3, 3 * c->N * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(c->stage + 3 * c->N, dg6, 6 * c->N * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return fail2(CSLBM_ECUDA, "copy to the device failed");
        gg = c->stage;
        dg = c->stage + 3 * c->N;
    }
    if (cslbm_status s = DISPATCH(c, metric)(c, gg, dg, c->gc)) return s;
    c->has_metric = 1;
    return CSLBM_OK;
}

cslbm_status cslbm2d_set_jacobian(cslbm2d_ctx* c, const double* J4, int on_device)
{
    if (!c || !J4) return fail2(CSLBM_EINVAL, "null argument");
    if (cudaMemcpyAsync(c->J, J4, 4 * c->N * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess)
        return fail2(CSLBM_ECUDA, "copy failed");
    return launched(c, "set_jacobian", !on_device);
}

cslbm_status cslbm2d_update_metric(cslbm2d_ctx* c, const double* g3, const double* dg6, const double* Jnew4,
                                   int on_device)
{
    if (!c || !g3 || !dg6 || !Jnew4) return fail2(CSLBM_EINVAL, "null argument");
    if (!c->has_state) return fail2(CSLBM_ESTATE, "update_metric before init_equilibrium");
    const double *gg, *dg, *Jn;
    if (on_device) {
        gg = g3;
        dg = dg6;
        Jn = Jnew4;
    } else {
        if (cudaMemcpyAsync(c->stage, g3, 3 * c->N * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(c->stage + 3 * c->N, dg6, 6 * c->N * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return fail2(CSLBM_ECUDA, "copy to the device failed");
        gg = c->stage;
        dg = c->stage + 3 * c->N;
        Jn = nullptr;
    }
    if (cslbm_status s = DISPATCH(c, metric)(c, gg, dg, 1 - c->gc)) return s;
    if (!on_device) {  // the staging area is free again: the Jacobian goes there
        if (cudaMemcpyAsync(c->stage, Jnew4, 4 * c->N * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return fail2(CSLBM_ECUDA, "copy to the device failed");
        Jn = c->stage;
    }
    if (cslbm_status s = DISPATCH(c, transform)(c, Jn)) return s;
    if (cudaMemcpyAsync(c->J, Jn, 4 * c->N * 8, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        return fail2(CSLBM_ECUDA, "copy failed");
    c->pc ^= 1;
    c->gc ^= 1;
    return launched(c, "update_metric", !on_device);
}

cslbm_status cslbm2d_set_boundary_velocity(cslbm2d_ctx* c, int axis, int side, const double* u2, int on_device)
{
    if (!c || axis < 0 || axis > 1 || side < 0 || side > 1) return fail2(CSLBM_EINVAL, "bad argument");
    if ((side ? c->p.bc_hi[axis] : c->p.bc_lo[axis]) == PER) return fail2(CSLBM_EINVAL, "periodic face");
    const int k = axis * 2 + side, nf = c->p.n[1 - axis];
    size_t off[12];
    layout(&c->p, off);
    double* base = (double*)((char*)c->P[0] - off[0] + off[8]);
    // faces packed as (axis 0: lo, hi of n1 nodes each) then (axis 1: lo, hi of n0)
    const size_t pos = axis == 0 ? (size_t)side * 2 * c->p.n[1] : (size_t)4 * c->p.n[1] + (size_t)side * 2 * c->p.n[0];
    double* dst = base + pos;
    if (!u2) {
        c->face[k] = nullptr;
        return CSLBM_OK;
    }
    if (cudaMemcpyAsync(dst, u2, 2 * (size_t)nf * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess)
        return fail2(CSLBM_ECUDA, "copy failed");
    c->face[k] = dst;
    return launched(c, "set_boundary_velocity", !on_device);
}

cslbm_status cslbm2d_init_equilibrium(cslbm2d_ctx* c, const double* rho, const double* u2, int on_device)
{
    if (!c) return fail2(CSLBM_EINVAL, "null argument");
    if (!c->has_metric) return fail2(CSLBM_ESTATE, "init before set_metric");
    const double *r = nullptr, *u = nullptr;
    if (rho) {
        if (cslbm_status s = in64(c, rho, c->N, on_device, &r)) return s;
    }
    if (u2) {
        if (on_device) u = u2;
        else {
            if (cudaMemcpyAsync(c->stage + c->N, u2, 2 * c->N * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
                return fail2(CSLBM_ECUDA, "copy failed");
            u = c->stage + c->N;
        }
    }
    if (c->r == 8) init<double>(c, r, u);
    else init<float>(c, r, u);
    c->has_state = 1;
    return launched(c, "init", !on_device);
}

cslbm_status cslbm2d_step(cslbm2d_ctx* c, int nsteps)
{
    if (!c || nsteps < 0) return fail2(CSLBM_EINVAL, "bad argument");
    if (!c->has_state) return fail2(CSLBM_ESTATE, "step before init_equilibrium");
    for (int t = 0; t < nsteps; t++) {
        if (c->r == 8) step_once<double>(c);
        else step_once<float>(c);
    }
    return launched(c, "step");
}

cslbm_status cslbm2d_get_moments(cslbm2d_ctx* c, double* rho, double* u2, int cartesian, int on_device)
{
    if (!c || !rho || !u2) return fail2(CSLBM_EINVAL, "null argument");
    if (!c->has_state) return fail2(CSLBM_ESTATE, "no state");
    double* r = rho;
    double* u = u2;
    if (!on_device) {
        r = c->stage;
        u = c->stage + c->N;
    }
    const Lat L = lat_of(c);
    if (c->r == 8)
        k2_readout<double><<<nb(c->N), TB, 0, c->stream>>>(L, (const double*)c->P[c->pc], (const double*)c->F[c->pc],
                                                           (const double*)c->G[c->gc], c->J, r, u, cartesian);
    else
        k2_readout<float><<<nb(c->N), TB, 0, c->stream>>>(L, (const float*)c->P[c->pc], (const float*)c->F[c->pc],
                                                          (const float*)c->G[c->gc], c->J, r, u, cartesian);
    if (!on_device) {
        if (cudaMemcpyAsync(rho, r, c->N * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(u2, u, 2 * c->N * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            return fail2(CSLBM_ECUDA, "copy failed");
    }
    return launched(c, "readout", true);
}

cslbm_status cslbm2d_total_mass(cslbm2d_ctx* c, double* out)
{
    if (!c || !out) return fail2(CSLBM_EINVAL, "null argument");
    if (!c->has_state) return fail2(CSLBM_ESTATE, "no state");
    cudaMemsetAsync(c->scratch, 0, 8, c->stream);
    const Lat L = lat_of(c);
    if (c->r == 8)
        k2_mass<double><<<nb(c->N), TB, 0, c->stream>>>(L, (const double*)c->P[c->pc], (const double*)c->F[c->pc],
                                                        (const double*)c->G[c->gc], c->scratch);
    else
        k2_mass<float><<<nb(c->N), TB, 0, c->stream>>>(L, (const float*)c->P[c->pc], (const float*)c->F[c->pc],
                                                       (const float*)c->G[c->gc], c->scratch);
    cudaMemcpyAsync(out, c->scratch, 8, cudaMemcpyDeviceToHost, c->stream);
    return launched(c, "mass", true);
}

cslbm_status cslbm2d_wall_force(cslbm2d_ctx* c, int axis, int side, double out2[2])
{
    if (!c || !out2 || axis < 0 || axis > 1 || side < 0 || side > 1) return fail2(CSLBM_EINVAL, "bad argument");
    if (!c->has_state) return fail2(CSLBM_ESTATE, "no state");
    cudaMemsetAsync(c->scratch, 0, 16, c->stream);
    const Lat L = lat_of(c);
    const long long nf = c->p.n[1 - axis];
    if (c->r == 8)
        k2_wall_force<double><<<nb(nf), TB, 0, c->stream>>>(L, (const double*)c->P[c->pc], (const double*)c->F[c->pc],
                                                            (const double*)c->G[c->gc], c->J, axis, side, c->scratch);
    else
        k2_wall_force<float><<<nb(nf), TB, 0, c->stream>>>(L, (const float*)c->P[c->pc], (const float*)c->F[c->pc],
                                                           (const float*)c->G[c->gc], c->J, axis, side, c->scratch);
    cudaMemcpyAsync(out2, c->scratch, 16, cudaMemcpyDeviceToHost, c->stream);
    return launched(c, "wall force", true);
}

}  // extern "C"
