// Arithmetic of one LBM step written for a value type T that is either one
// node's scalar (float / double) or a pair of x-adjacent nodes (Pair<float>,
// Pair<double>).  For Pair<float> every operation is one packed FP32
// instruction (FADD2 / FMUL2 / FFMA2), so a thread steps two nodes for the
// instruction count of one.
//
// The D3Q19 populations come in opposite pairs (l, l+1) for odd l, which the
// sums and the Hermite recomposition exploit: with p = s_l + s_l+1 and
// q = s_l - s_l+1 the even moments need only p and the odd ones only q, and
// the recomposed values of l and l+1 share their even part and differ in the
// sign of the odd part.
#pragma once

#include "lbm_device.cuh"

namespace cslbm {

template <class R> struct Pair;

template <> struct Pair<float> {
    float2 v;
    __device__ __forceinline__ Pair() {}
    __device__ __forceinline__ Pair(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ Pair(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit Pair(float2 x) : v(x) {}
    __device__ __forceinline__ float lo() const { return v.x; }
    __device__ __forceinline__ float hi() const { return v.y; }
};
__device__ __forceinline__ Pair<float> operator+(Pair<float> a, Pair<float> b) { return Pair<float>(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ Pair<float> operator-(Pair<float> a, Pair<float> b)
{
    return Pair<float>(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y)));
}
__device__ __forceinline__ Pair<float> operator*(Pair<float> a, Pair<float> b) { return Pair<float>(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ Pair<float> fmad(Pair<float> a, Pair<float> b, Pair<float> c)
{
    return Pair<float>(__ffma2_rn(a.v, b.v, c.v));
}
__device__ __forceinline__ Pair<float> recip(Pair<float> a) { return Pair<float>(1.0f / a.v.x, 1.0f / a.v.y); }

template <> struct Pair<double> {
    double x, y;
    __device__ __forceinline__ Pair() {}
    __device__ __forceinline__ Pair(double a) : x(a), y(a) {}
    __device__ __forceinline__ Pair(double a, double b) : x(a), y(b) {}
    __device__ __forceinline__ double lo() const { return x; }
    __device__ __forceinline__ double hi() const { return y; }
};
__device__ __forceinline__ Pair<double> operator+(Pair<double> a, Pair<double> b) { return Pair<double>(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ Pair<double> operator-(Pair<double> a, Pair<double> b) { return Pair<double>(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ Pair<double> operator*(Pair<double> a, Pair<double> b) { return Pair<double>(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ Pair<double> fmad(Pair<double> a, Pair<double> b, Pair<double> c)
{
    return Pair<double>(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ Pair<double> recip(Pair<double> a) { return Pair<double>(1.0 / a.x, 1.0 / a.y); }

__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float recip(float a) { return 1.0f / a; }
__device__ __forceinline__ double recip(double a) { return 1.0 / a; }

// ---------------------------------------------------------------------------
// moments of the shifted populations s = h - w:
//   m0 = sum s, m1 = sum s c, m2 = sum s c c (packed 00,01,02,11,12,22)
// ---------------------------------------------------------------------------
template <class T> struct PairSums {
    T p[9], q[9];  // s_l + s_l+1 and s_l - s_l+1 for l = 1, 3, ..., 17
};

template <class T>
__device__ __forceinline__ void pair_sums(const T s[Q], PairSums<T>& P)
{
#pragma unroll
    for (int k = 0; k < 9; k++) {
        P.p[k] = s[2 * k + 1] + s[2 * k + 2];
        P.q[k] = s[2 * k + 1] - s[2 * k + 2];
    }
}

// first moment from the odd parts (c of l = 2k+1: k=0 +x, 1 +y, 2 +z,
// 3 (1,1,0), 4 (1,-1,0), 5 (1,0,1), 6 (1,0,-1), 7 (0,1,1), 8 (0,1,-1))
template <class T>
__device__ __forceinline__ void first_moment(const PairSums<T>& P, T m1[3])
{
    m1[0] = ((P.q[0] + P.q[3]) + (P.q[4] + P.q[5])) + P.q[6];
    m1[1] = ((P.q[1] + P.q[3]) - (P.q[4] - P.q[7])) + P.q[8];
    m1[2] = ((P.q[2] + P.q[5]) - (P.q[6] - P.q[7])) - P.q[8];
}

template <class T>
__device__ __forceinline__ void all_moments(const T s[Q], const PairSums<T>& P, T& m0, T m1[3], T m2[6])
{
    const T exy = P.p[3] + P.p[4], exz = P.p[5] + P.p[6], eyz = P.p[7] + P.p[8];
    m0 = s[0] + ((P.p[0] + P.p[1]) + P.p[2]) + ((exy + exz) + eyz);
    first_moment(P, m1);
    m2[0] = P.p[0] + (exy + exz);
    m2[3] = P.p[1] + (exy + eyz);
    m2[5] = P.p[2] + (exz + eyz);
    m2[1] = P.p[3] - P.p[4];
    m2[2] = P.p[5] - P.p[6];
    m2[4] = P.p[7] - P.p[8];
}

// ---------------------------------------------------------------------------
// Lattice gradient D[k][i] = 1/c_s^2 sum_l w_l c_l^k j^i(x + c_l) (App. D),
// from the differences d_l^i = j^i(x + c_l) - j^i(x - c_l) of the nine
// opposite pairs (same ordering as PairSums): faces weigh 3/18, edges 3/36.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void gradient_from_pairs(const T d[9][3], T D[3][3])
{
    const T wf(1.0 / 6.0), we(1.0 / 12.0);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        D[0][i] = fmad(we, ((d[3][i] + d[4][i]) + (d[5][i] + d[6][i])), wf * d[0][i]);
        D[1][i] = fmad(we, ((d[3][i] - d[4][i]) + (d[7][i] + d[8][i])), wf * d[1][i]);
        D[2][i] = fmad(we, ((d[5][i] - d[6][i]) + (d[7][i] - d[8][i])), wf * d[2][i]);
    }
}

// ---------------------------------------------------------------------------
// stress, forcing moments and collision coefficients (as in kernels.cuh, in
// explicit fused multiply-adds)
// ---------------------------------------------------------------------------
template <class T> struct GeoT {
    T sg, isg, gi[6], gam[18], gc[3];
};
template <class T> struct HistT {
    T A, B[3], C[6];
};

// T = Pi^eq + (1 - 1/2tau)(Pi - Pi^eq), Pi^eq = rho theta g^-1 + j j / rho,
// Pi = sqrt(g)(c_s^2 delta + m2) + C'/2    (Eq. fields3, App. B)
template <class T, class R>
__device__ __forceinline__ void stress_t(R theta, R kvisc, const GeoT<T>& G, T rho, T ir, const T j[3],
                                         const T m2[6], const HistT<T>& Hp, T Tt[6])
{
    const T rt = rho * T(theta), half(0.5), third(1.0 / 3.0), kv(kvisc);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++) {
            const int k = s6(a, b);
            const T pieq = fmad(j[a] * j[b], ir, rt * G.gi[k]);
            const T pi = fmad(G.sg, (a == b ? m2[k] + third : m2[k]), half * Hp.C[k]);
            Tt[k] = fmad(kv, pi - pieq, pieq);
        }
}

// Eqs. forcing-A/B/C with gc_k = Gamma^j_kj:
//   A = -2 gc.j,  B^i = F^i - 2 gc_j T^ij - Gamma^i_jk T^jk,
//   C^ij = c_s^2 (dbar_j j^i + dbar_i j^j + delta^ij dbar_k j^k)
//        - theta (g^jk nabla_k j^i + g^ik nabla_k j^j + g^ij nabla_k j^k)
template <class T, class R>
__device__ __forceinline__ void forcing_t(R theta, const R fext[3], const GeoT<T>& G, const T j[3], const T Tt[6],
                                          const T D[3][3], HistT<T>& H)
{
    const T two(2), m2(-2);
    H.A = m2 * fmad(G.gc[0], j[0], fmad(G.gc[1], j[1], G.gc[2] * j[2]));
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int o = i * 6;
        // Gamma^i_jk T^jk over the symmetric pair (j,k)
        T g = fmad(G.gam[o + 0], Tt[0], fmad(G.gam[o + 3], Tt[3], G.gam[o + 5] * Tt[5]));
        g = fmad(two, fmad(G.gam[o + 1], Tt[1], fmad(G.gam[o + 2], Tt[2], G.gam[o + 4] * Tt[4])), g);
        const T gt = fmad(G.gc[0], Tt[s6(i, 0)], fmad(G.gc[1], Tt[s6(i, 1)], G.gc[2] * Tt[s6(i, 2)]));
        H.B[i] = (T(fext[i]) - g) - two * gt;
    }
    T bard[3][3], cov[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int i = 0; i < 3; i++) {
            bard[k][i] = D[k][i] - G.gc[k] * j[i];
            cov[k][i] = fmad(G.gam[i * 6 + s6(k, 0)], j[0],
                             fmad(G.gam[i * 6 + s6(k, 1)], j[1], fmad(G.gam[i * 6 + s6(k, 2)], j[2], D[k][i])));
        }
    const T divbar = (bard[0][0] + bard[1][1]) + bard[2][2];
    const T divcov = (cov[0][0] + cov[1][1]) + cov[2][2];
    const T cs2(1.0 / 3.0), th(theta);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int jj = i; jj < 3; jj++) {
            T c = bard[jj][i] + bard[i][jj];
            if (i == jj) c = c + divbar;
            T t = G.gi[s6(i, jj)] * divcov;
#pragma unroll
            for (int k = 0; k < 3; k++) t = fmad(G.gi[s6(jj, k)], cov[k][i], fmad(G.gi[s6(i, k)], cov[k][jj], t));
            H.C[s6(i, jj)] = fmad(cs2, c, T(-theta) * t);
        }
}

// Collision (Eq. collision) for the stored form s = h - w with h = f - F'/2:
//   s*_l = (1 - w) s_l + w_l d0 + w_l/sqrt(g) [3 E1.c_l + 9/2 (E2:c_l c_l - tr E2/3)]
//   d0 = w m0 + A/sqrt g,  E1 = w j + B - w/2 B',  E2 = w a2^eq + b2 - w/2 b2'
template <class T, class R>
__device__ __forceinline__ void collide_t(R omega, R theta, const GeoT<T>& G, const T s[Q], T m0, T rho, T ir,
                                          const T j[3], const HistT<T>& Hp, const HistT<T>& H, T out[Q])
{
    const T om(omega), hom(0.5 * omega), third(1.0 / 3.0);
    T E1[3], E2[6];
#pragma unroll
    for (int a = 0; a < 3; a++) E1[a] = fmad(om, j[a], H.B[a] - hom * Hp.B[a]);
    const T rt = rho * T(theta), r3 = rho * third, A3 = H.A * third, Ap3 = Hp.A * third;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++) {
            const int k = s6(a, b);
            T a2 = fmad(j[a] * j[b], ir, rt * G.gi[k]);
            T b2 = H.C[k], b2p = Hp.C[k];
            if (a == b) {
                a2 = a2 - r3;
                b2 = b2 - A3;
                b2p = b2p - Ap3;
            }
            E2[k] = fmad(om, a2, b2 - hom * b2p);
        }
    const T d0 = fmad(om, m0, H.A * G.isg);
    const T t = T(1.5) * ((E2[0] + E2[3]) + E2[5]);
    const T one_m(1.0 - omega);
    // rest: w0 [d0 + isg (-t)]
    out[0] = fmad(one_m, s[0], T(1.0 / 3.0) * fmad(G.isg, T(0) - t, d0));
    // faces: even 9/2 E2_aa - t, odd 3 E1_a
    const T wf(1.0 / 18.0), we(1.0 / 36.0);
    const T fd0 = wf * d0, fis = wf * G.isg, ed0 = we * d0, eis = we * G.isg;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const T ev = fmad(T(4.5), E2[s6(a, a)], T(0) - t), od = T(3) * E1[a];
        out[2 * a + 1] = fmad(fis, ev + od, fmad(one_m, s[2 * a + 1], fd0));
        out[2 * a + 2] = fmad(fis, ev - od, fmad(one_m, s[2 * a + 2], fd0));
    }
    // edges in the (a, b) planes: c = (+a,+b), (-a,-b), (+a,-b), (-a,+b)
    const int ea[3] = {0, 0, 1}, eb[3] = {1, 2, 2};
#pragma unroll
    for (int e = 0; e < 3; e++) {
        const int a = ea[e], b = eb[e], l = 7 + 4 * e;
        const T sab = fmad(T(4.5), E2[s6(a, a)] + E2[s6(b, b)], T(0) - t), dab = T(9) * E2[s6(a, b)];
        const T evp = sab + dab, evm = sab - dab;
        const T odp = T(3) * (E1[a] + E1[b]), odm = T(3) * (E1[a] - E1[b]);
        out[l] = fmad(eis, evp + odp, fmad(one_m, s[l], ed0));
        out[l + 1] = fmad(eis, evp - odp, fmad(one_m, s[l + 1], ed0));
        out[l + 2] = fmad(eis, evm + odm, fmad(one_m, s[l + 2], ed0));
        out[l + 3] = fmad(eis, evm - odm, fmad(one_m, s[l + 3], ed0));
    }
}

}  // namespace cslbm
