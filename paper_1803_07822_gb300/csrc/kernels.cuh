// Kernels of the curved-space D3Q19 step, templated on the storage type S
// of the populations and the compute type R.  Included once per storage
// format by the inst_*.cu units, which instantiate the ops table.
#pragma once

#include <type_traits>

#include "ctx.h"
#include "flat_step.cuh"
#include "fused_rows.cuh"
#include "lbm_device.cuh"
#include "fp_convert.h"
#include "make_lat.h"

namespace cslbm {

constexpr int TPB = 256;

inline unsigned nblocks(long long n) { return (unsigned)((n + TPB - 1) / TPB); }

__device__ __forceinline__ void node_coords(const Lat& L, long long v, int& x, int& y, int& z)
{
    x = (int)(v % L.n[0]);
    long long r = v / L.n[0];
    y = (int)(r % L.n[1]);
    z = (int)(r / L.n[1]);
}

// ---------------------------------------------------------------------------
// Metric update (App. A): inverse metric by cofactors in FP64, sqrt(det g),
// then Gamma^i_jk = 1/2 g^il (d_j g_kl + d_k g_jl - d_l g_jk) in R.
// ---------------------------------------------------------------------------
// a double rounded to the compute type (FP32 on the integer units)
template <class R> __device__ __forceinline__ R to_real(double x);
template <> __device__ __forceinline__ float to_real<float>(double x) { return f64_to_f32_rn(x); }
template <> __device__ __forceinline__ double to_real<double>(double x) { return x; }
// FP32 inputs (the mixed-precision chart change) are taken as they are
template <class R> __device__ __forceinline__ R to_real(float x) { return R(x); }

// geometry of node v (G[.][v]: sqrt(g), g^ij, Gamma) from its metric g6 /
// dg18 at entry t of the inputs (stride apart); returns false for det g <= 0
template <class R, class DT = double>
__device__ __forceinline__ bool metric_node(const double* __restrict__ g6, const DT* __restrict__ dg18,
                                            long long stride, long long t, R* __restrict__ geo, long long N,
                                            long long v, R& sg_out)
{
    const double a = g6[0 * stride + t], b = g6[1 * stride + t], c = g6[2 * stride + t];
    const double d = g6[3 * stride + t], e = g6[4 * stride + t], f = g6[5 * stride + t];
    // g = [[a b c] [b d e] [c e f]]
    const double A = d * f - e * e, B = c * e - b * f, C = b * e - c * d;
    const double det = a * A + b * B + c * C;
    if (!(det > 0.0)) return false;
    // 1/det and sqrt(det) in FP64.  For FP32-and-narrower storage they start
    // from FP32 estimates refined by one Newton step each (relative error
    // ~1e-14 before the rounding to R), which spares the FP64 divide and
    // square root; FP64 storage divides exactly.  The conversions between
    // FP64 and FP32 run on the integer units (fp_convert.h): as FP64-pipe
    // instructions they were most of this kernel's time.
    double id, sd;
    if constexpr (std::is_same<R, double>::value) {
        id = 1.0 / det;
        sd = sqrt(det);
    } else {
        // 1e-30 < det < 1e30, compared on the bit patterns of positive doubles
        const long long bits = __double_as_longlong(det);
        if (bits > 0x39B4484BFEEBC2A0ll && bits < 0x46293E5939A08CEAll) {
            const float df = f64_to_f32_rn(det);
            const double r0 = f32_to_f64(__frcp_rn(df));
            id = fma(r0, fma(-det, r0, 1.0), r0);        // r0 (2 - det r0)
            const double y0 = f32_to_f64(rsqrtf(df));    // ~ 1/sqrt(det)
            const double s0 = det * y0;
            sd = fma(0.5 * y0, fma(-s0, s0, det), s0);   // s0 + (det - s0^2) / (2 s0)
        } else {
            id = 1.0 / det;
            sd = sqrt(det);
        }
    }
    double gi[6] = {A * id, B * id, C * id, (a * f - c * c) * id, (b * c - a * e) * id, (a * d - b * b) * id};
    R dg[3][6], gr[6];
#pragma unroll
    for (int m = 0; m < 6; m++) gr[m] = to_real<R>(gi[m]);
    sg_out = to_real<R>(sd);
    geo[v] = sg_out;
#pragma unroll
    for (int k = 0; k < 6; k++) geo[(1 + k) * N + v] = gr[k];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int m = 0; m < 6; m++) dg[k][m] = to_real<R>(dg18[(k * 6 + m) * stride + t]);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int k = j; k < 3; k++) {
                R s = R(0);
#pragma unroll
                for (int l = 0; l < 3; l++) s += gr[s6(i, l)] * (dg[j][s6(k, l)] + dg[k][s6(j, l)] - dg[l][s6(j, k)]);
                geo[(7 + i * 6 + s6(j, k)) * N + v] = R(0.5) * s;
            }
    return true;
}

template <class R>
__global__ void __launch_bounds__(TPB) k_metric(const double* __restrict__ g6, const double* __restrict__ dg18,
                                                long long stride, long long v0, long long cnt, R* __restrict__ geo,
                                                long long N, int* bad)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    R sg;
    if (!metric_node<R>(g6, dg18, stride, t, geo, N, v0 + t, sg)) atomicOr(bad, 1);
}

// ---------------------------------------------------------------------------
// Initial state: the slots of P that node x's populations will be read from
// get f^eq_l(x) - w_l (history still zero, so h = f).
// ---------------------------------------------------------------------------
template <class S, class R>
__global__ void __launch_bounds__(TPB) k_init_scatter(Lat L, const double* __restrict__ rho0, const double* __restrict__ u0,
                                                      long long stride, long long v0, long long cnt,
                                                      const R* __restrict__ geo, S* __restrict__ P)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    long long v = v0 + t;
    int x, y, z;
    node_coords(L, v, x, y, z);
    Geo<R> G;
    load_metric(geo, L.N, v, G);
    R rho = rho0 ? R(rho0[t]) : R(1);
    R j[3];
#pragma unroll
    for (int a = 0; a < 3; a++) j[a] = u0 ? rho * R(u0[a * stride + t]) : R(0);
    R a2[6];
    feq_coeffs(rho, j, G.gi, R(L.theta), a2);
    const R tr = a2[0] + a2[3] + a2[5];
    const R b0 = rho - G.sg;  // f^eq - w = w/sqrt(g) [(rho - sqrt g) + ...]
#pragma unroll
    for (int l = 0; l < Q; l++) {
        int r[3] = {x - cvec(l, 0), y - cvec(l, 1), z - cvec(l, 2)};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (r[a] < 0 || r[a] >= L.n[a]) {
                if ((r[a] < 0 ? L.bclo[a] : L.bchi[a]) == BC_PERIODIC) r[a] = wrapc(r[a], L.n[a]);
                else ok = false;
            }
        }
        if (ok) Store<S>::st(P + (long long)pslot(l) * L.N + nidx(L, r[0], r[1], r[2]), hermite_l(l, G.isg, b0, j, a2, tr));
    }
}

// P slots -= F_l(x)/2: the stored h = f - F(t - dt)/2 once the history exists.
template <class S, class R>
__global__ void __launch_bounds__(TPB) k_half_shift(Lat L, S* __restrict__ P, const R* __restrict__ hist,
                                                    const R* __restrict__ geo)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= L.N) return;
    int x, y, z;
    node_coords(L, v, x, y, z);
    Hist<R> H;
    load_hist(hist, L.N, v, H);
    const R isg = R(1) / geo[v];
#pragma unroll
    for (int l = 0; l < Q; l++) {
        int r[3] = {x - cvec(l, 0), y - cvec(l, 1), z - cvec(l, 2)};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (r[a] < 0 || r[a] >= L.n[a]) {
                if ((r[a] < 0 ? L.bclo[a] : L.bchi[a]) == BC_PERIODIC) r[a] = wrapc(r[a], L.n[a]);
                else ok = false;
            }
        }
        if (ok) {
            S* p = P + (long long)pslot(l) * L.N + nidx(L, r[0], r[1], r[2]);
            Store<S>::st(p, Store<S>::ld(p) - R(0.5) * forcing_l(l, isg, H));
        }
    }
}

// macroscopic fields of a node from its (boundary-filled) populations
template <class S, class R> struct NodeMoments {
    R s[Q];
    R m0, m1[3], m2[6];
    R rho, j[3];
    Hist<R> Hp;
};

template <class S, class R>
__device__ __forceinline__ void node_moments(const Lat& L, const S* __restrict__ P, const R* __restrict__ hist,
                                             const R* __restrict__ geo, int x, int y, int z, long long v, R sg,
                                             NodeMoments<S, R>& M)
{
    node_pops<S, R>(L, P, hist, geo, x, y, z, M.s);
    load_hist(hist, L.N, v, M.Hp);
    sums(M.s, M.m0, M.m1, M.m2);
    M.rho = sg * (R(1) + M.m0) + R(0.5) * M.Hp.A;
#pragma unroll
    for (int a = 0; a < 3; a++) M.j[a] = sg * M.m1[a] + R(0.5) * M.Hp.B[a];
}

// ---------------------------------------------------------------------------
// Pieces of the step used by the initial forcing pass.
// ---------------------------------------------------------------------------
// T = Pi^eq + (1 - 1/2tau)(Pi - Pi^eq), Pi^eq = rho theta g^-1 + j j / rho,
// Pi = sqrt(g)(c_s^2 delta + m2) + C'/2    (Eq. fields3, App. B)
template <class R>
__device__ __forceinline__ void stress(const Lat& L, const Geo<R>& G, R rho, const R j[3], const R m2[6],
                                       const Hist<R>& Hp, R T[6])
{
    const R ir = R(1) / rho, theta = R(L.theta), kv = R(L.kvisc);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++) {
            const int k = s6(a, b);
            R pieq = rho * theta * G.gi[k] + j[a] * j[b] * ir;
            R pi = G.sg * ((a == b ? R(1.0 / 3.0) : R(0)) + m2[k]) + R(0.5) * Hp.C[k];
            T[k] = pieq + kv * (pi - pieq);
        }
}

// Collision (Eq. collision) written for the stored form s = h - w, with
// h = f - F'/2:  f* = (1 - w) h + w f^eq + F - w/2 F'  (w = 1/tau), i.e.
//   s* = (1 - w) s + w_l (w m0 + A/sqrt g) + Hermite_l(0, E1, E2),
//   E1 = w j + B - w/2 B',  E2 = w a2^eq + b2 - w/2 b2'.
template <class R>
__device__ __forceinline__ void collide_coeffs(const Lat& L, const Geo<R>& G, R m0, R rho, const R j[3],
                                               const Hist<R>& Hp, const Hist<R>& H, R& d0, R E1[3], R E2[6], R& trE2)
{
    const R om = R(L.omega);
    R a2[6];
    feq_coeffs(rho, j, G.gi, R(L.theta), a2);
#pragma unroll
    for (int a = 0; a < 3; a++) E1[a] = om * j[a] + H.B[a] - R(0.5) * om * Hp.B[a];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const bool dia = (k == 0 || k == 3 || k == 5);
        R b2 = H.C[k] - (dia ? H.A * R(1.0 / 3.0) : R(0));
        R b2p = Hp.C[k] - (dia ? Hp.A * R(1.0 / 3.0) : R(0));
        E2[k] = om * a2[k] + b2 - R(0.5) * om * b2p;
    }
    trE2 = E2[0] + E2[3] + E2[5];
    d0 = om * m0 + H.A * G.isg;
}

template <class R>
__device__ __forceinline__ void store_hist(R* __restrict__ h, long long N, long long v, const Hist<R>& H)
{
    h[v] = H.A;
#pragma unroll
    for (int a = 0; a < 3; a++) h[(1 + a) * N + v] = H.B[a];
#pragma unroll
    for (int a = 0; a < 6; a++) h[(4 + a) * N + v] = H.C[a];
}

// Forcing coefficients of the current state (used once, at initialisation,
// to set F(x, -dt) := F(x, 0)); the gradient reads the momentum field jf.
template <class S, class R>
__global__ void __launch_bounds__(TPB) k_forcing(Lat L, const S* __restrict__ P, const R* __restrict__ hin,
                                                 R* __restrict__ hout, const R* __restrict__ geo,
                                                 const void* __restrict__ jfv)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= L.N) return;
    const Mom4<R>* jf = (const Mom4<R>*)jfv;
    int x, y, z;
    node_coords(L, v, x, y, z);
    Geo<R> G;
    load_geo(geo, L.N, v, G);
    NodeMoments<S, R> M;
    node_moments<S, R>(L, P, hin, geo, x, y, z, v, G.sg, M);
    R T[6];
    stress(L, G, M.rho, M.j, M.m2, M.Hp, T);
    // lattice gradient D[k][i] = 1/c_s^2 sum_l w_l c_l^k j^i(x + c_l) (App. D)
    R D[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int i = 0; i < 3; i++) D[k][i] = R(0);
#pragma unroll
    for (int l = 1; l < Q; l++) {
        const int cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
        const R wl = R(3.0 * wq(l));
        const Mom4<R> jn = mom_site<R>(L, jf, x + cx, y + cy, z + cz);
        const R jv[3] = {jn.x, jn.y, jn.z};
#pragma unroll
        for (int i = 0; i < 3; i++) {
            D[0][i] += (wl * cx) * jv[i];
            D[1][i] += (wl * cy) * jv[i];
            D[2][i] += (wl * cz) * jv[i];
        }
    }
    Hist<R> H;
    forcing_moments(L, G, M.j, T, D, H);
    store_hist(hout, L.N, v, H);
}

// ---------------------------------------------------------------------------
// Chart change (Sec. IV.B), node-wise: D phi = Jnew^-1 Jold; a_(0) kept,
// a_(1) -> D a_(1), Pi -> D Pi D^T (or a_(2) -> D a_(2) D^T), recomposed with
// the new sqrt(g); the history's A, B, C as scalar, vector, rank-2 tensor.
// Writes the transformed state into the other buffers (same pull slots).
// ---------------------------------------------------------------------------
// The tensor transformation with D phi = Dp and the recomposition with the
// new sqrt(g) of one node's f-moments (rho, j, M2 = Pi or a_(2)) and history
// (A, B and Cs = C, or b_(2) = C - c_s^2 delta A with literal), stored into
// the pull slots and history of node (x, y, z) = v.
template <class S, class R>
__device__ __forceinline__ void transform_store(const Lat& L, S* __restrict__ Pout, R* __restrict__ hout, R sgn,
                                                int x, int y, int z, long long v, const R (&Dp)[3][3], R rho,
                                                const R (&j)[3], const R (&M2)[6], R A, const R (&B)[3],
                                                const R (&Cs)[6], int literal)
{
    auto vec = [&](const R in[3], R out[3]) {
#pragma unroll
        for (int i = 0; i < 3; i++) out[i] = Dp[i][0] * in[0] + Dp[i][1] * in[1] + Dp[i][2] * in[2];
    };
    auto ten = [&](const R in[6], R out[6]) {
        R tmp[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int m = 0; m < 3; m++)
                tmp[i][m] = Dp[i][0] * in[s6(0, m)] + Dp[i][1] * in[s6(1, m)] + Dp[i][2] * in[s6(2, m)];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = i; k < 3; k++) out[s6(i, k)] = tmp[i][0] * Dp[k][0] + tmp[i][1] * Dp[k][1] + tmp[i][2] * Dp[k][2];
    };
    R j2[3], P2[6];
    vec(j, j2);
    ten(M2, P2);
    if (!literal) {
        P2[0] -= rho * R(1.0 / 3.0);
        P2[3] -= rho * R(1.0 / 3.0);
        P2[5] -= rho * R(1.0 / 3.0);
    }
    // history: A scalar, B vector, C (or, with literal, b_(2) = C - c_s^2 delta A) rank 2
    Hist<R> Hn;
    Hn.A = A;
    vec(B, Hn.B);
    ten(Cs, Hn.C);
    if (literal) {
        Hn.C[0] += Hn.A * R(1.0 / 3.0);
        Hn.C[3] += Hn.A * R(1.0 / 3.0);
        Hn.C[5] += Hn.A * R(1.0 / 3.0);
    }
    const R isgn = R(1) / sgn;
    hout[v] = Hn.A;
#pragma unroll
    for (int a = 0; a < 3; a++) hout[(1 + a) * L.N + v] = Hn.B[a];
#pragma unroll
    for (int a = 0; a < 6; a++) hout[(4 + a) * L.N + v] = Hn.C[a];
    // f~ - F~/2 - w with f~ - w = w/sqrt(g~) P_l(rho - sqrt g~, j~, Pi~ - c_s^2 rho delta) and
    // F~ = w/sqrt(g~) P_l(A, B, C - c_s^2 delta A): one expansion of the difference
    R b1[3], b2[6];
    const R b0 = rho - sgn - R(0.5) * Hn.A;
#pragma unroll
    for (int a = 0; a < 3; a++) b1[a] = j2[a] - R(0.5) * Hn.B[a];
#pragma unroll
    for (int k = 0; k < 6; k++)
        b2[k] = P2[k] - R(0.5) * (Hn.C[k] - ((k == 0 || k == 3 || k == 5) ? Hn.A * R(1.0 / 3.0) : R(0)));
    const R trb2 = b2[0] + b2[3] + b2[5];
    // the slot of population l is that of the node r - c_l, which pulls it;
    // none past a non-periodic face.  Offsets of r - c per axis:
    const int r0[3] = {x, y, z};
    unsigned off[3][3], okm = 0u, stride = 1u;
#pragma unroll
    for (int a = 0; a < 3; a++) {
#pragma unroll
        for (int c = -1; c <= 1; c++) {
            int q = r0[a] - c;
            bool in = q >= 0 && q < L.n[a];
            if (!in && (q < 0 ? L.bclo[a] : L.bchi[a]) == BC_PERIODIC) {
                q = wrapc(q, L.n[a]);
                in = true;
            }
            off[a][c + 1] = in ? (unsigned)q * stride : 0u;
            okm |= in ? 1u << (3 * a + c + 1) : 0u;
        }
        stride *= (unsigned)L.n[a];
    }
#pragma unroll
    for (int l = 0; l < Q; l++) {
        const int cx = cvec(l, 0) + 1, cy = cvec(l, 1) + 1, cz = cvec(l, 2) + 1;
        const unsigned need = (1u << cx) | (1u << (3 + cy)) | (1u << (6 + cz));
        if ((okm & need) != need) continue;
        const R val = hermite_l(l, isgn, b0, b1, b2, trb2);
        Store<S>::st(Pout + (long long)pslot(l) * L.N + (off[2][cz] + off[1][cy] + off[0][cx]), val);
    }
}

// D phi = Jn^-1 Jo at the precision Cm of n and o (FP64 for FP64 storage,
// FP32 otherwise)
template <class Cm, class R>
__device__ __forceinline__ void dphi_of(const Cm (&n)[9], const Cm (&o)[9], R (&Dp)[3][3])
{
    Cm inv[9];
    {
        const Cm c00 = n[4] * n[8] - n[5] * n[7], c01 = n[5] * n[6] - n[3] * n[8], c02 = n[3] * n[7] - n[4] * n[6];
        const Cm det = n[0] * c00 + n[1] * c01 + n[2] * c02, id = Cm(1) / det;
        inv[0] = c00 * id;
        inv[3] = c01 * id;
        inv[6] = c02 * id;
        inv[1] = (n[2] * n[7] - n[1] * n[8]) * id;
        inv[4] = (n[0] * n[8] - n[2] * n[6]) * id;
        inv[7] = (n[1] * n[6] - n[0] * n[7]) * id;
        inv[2] = (n[1] * n[5] - n[2] * n[4]) * id;
        inv[5] = (n[2] * n[3] - n[0] * n[5]) * id;
        inv[8] = (n[0] * n[4] - n[1] * n[3]) * id;
    }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Cm s = Cm(0);
#pragma unroll
            for (int m = 0; m < 3; m++) s += inv[i * 3 + m] * o[m * 3 + k];
            Dp[i][k] = R(s);
        }
}

// the same from FP64 Jacobians, rounded to Cm first
template <class Cm, class R>
__device__ __forceinline__ void dphi(const double (&Jn)[9], const double (&Jo)[9], R (&Dp)[3][3])
{
    Cm n[9], o[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        n[k] = to_real<Cm>(Jn[k]);
        o[k] = to_real<Cm>(Jo[k]);
    }
    dphi_of<Cm, R>(n, o, Dp);
}

// the f-moments and history of a node in the form the transformation takes:
// out = {rho, j[3], M2[6], A, B[3], Cs[6]}
template <class S, class R>
__device__ __forceinline__ void transform_inputs(const Lat& L, const S* __restrict__ Pin, const R* __restrict__ hin,
                                                 const R* __restrict__ geo_old, int x, int y, int z, long long v,
                                                 int literal, R (&out)[20])
{
    const R sgo = geo_old[v];
    NodeMoments<S, R> M;
    node_moments<S, R>(L, Pin, hin, geo_old, x, y, z, v, sgo, M);
    out[0] = M.rho;
#pragma unroll
    for (int a = 0; a < 3; a++) out[1 + a] = M.j[a];
    // moments of f: a0 = rho, a1 = j, M2 = Pi (or a_(2))
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const bool dia = (k == 0 || k == 3 || k == 5);
        R m2 = sgo * ((dia ? R(1.0 / 3.0) : R(0)) + M.m2[k]) + R(0.5) * M.Hp.C[k];
        if (literal && dia) m2 -= M.rho * R(1.0 / 3.0);
        out[4 + k] = m2;
    }
    out[10] = M.Hp.A;
#pragma unroll
    for (int a = 0; a < 3; a++) out[11 + a] = M.Hp.B[a];
#pragma unroll
    for (int k = 0; k < 6; k++)
        out[14 + k] = M.Hp.C[k] - ((literal && (k == 0 || k == 3 || k == 5)) ? M.Hp.A * R(1.0 / 3.0) : R(0));
}

template <class S, class R>
__global__ void __launch_bounds__(TPB) k_transform(Lat L, const S* __restrict__ Pin, S* __restrict__ Pout,
                                                   const R* __restrict__ hin, R* __restrict__ hout,
                                                   const R* __restrict__ geo_old, const R* __restrict__ geo_new,
                                                   R* __restrict__ J, const double* __restrict__ Jnew,
                                                   long long stride, long long v0, long long cnt, int literal)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    long long v = v0 + t;
    int x, y, z;
    node_coords(L, v, x, y, z);
    R in[20];
    transform_inputs<S, R>(L, Pin, hin, geo_old, x, y, z, v, literal, in);
    // D phi = Jnew^-1 Jold at the precision of R (the stored Jacobian is kept
    // in R; the caller's FP64 Jnew is rounded to it and becomes the stored one)
    R Jo[9], Jn[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        Jo[k] = J[k * L.N + v];
        Jn[k] = to_real<R>(Jnew[k * stride + t]);
    }
    R Dp[3][3];
    dphi_of<R, R>(Jn, Jo, Dp);
#pragma unroll
    for (int k = 0; k < 9; k++) J[k * L.N + v] = Jn[k];
    const R j[3] = {in[1], in[2], in[3]}, B[3] = {in[11], in[12], in[13]};
    const R M2[6] = {in[4], in[5], in[6], in[7], in[8], in[9]};
    const R Cs[6] = {in[14], in[15], in[16], in[17], in[18], in[19]};
    transform_store<S, R>(L, Pout, hout, geo_new[v], x, y, z, v, Dp, in[0], j, M2, in[10], B, Cs, literal);
}

// The whole node-wise chart change in one pass (device inputs): the new
// geometry of the node from its metric (as k_metric), then the
// transformation of its state (as k_transform) with the new sqrt(g) from
// registers.  The metric's FP64 arithmetic overlaps the transformation's
// memory traffic instead of running as a pass of its own.
template <class S, class R, class DT = double>
__global__ void __launch_bounds__(TPB, 3) k_chart(Lat L, const S* __restrict__ Pin, S* __restrict__ Pout,
                                               const R* __restrict__ hin, R* __restrict__ hout,
                                               const R* __restrict__ geo_old, R* __restrict__ geo_new,
                                               R* __restrict__ J, const double* __restrict__ g6,
                                               const DT* __restrict__ dg18, const DT* __restrict__ Jnew,
                                               int literal, int* bad)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= L.N) return;
    R sgn;
    if (!metric_node<R, DT>(g6, dg18, L.N, v, geo_new, L.N, v, sgn)) {
        atomicOr(bad, 1);
        return;
    }
    int x, y, z;
    node_coords(L, v, x, y, z);
    R in[20];
    transform_inputs<S, R>(L, Pin, hin, geo_old, x, y, z, v, literal, in);
    R Jo[9], Jn[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        Jo[k] = J[k * L.N + v];
        Jn[k] = to_real<R>(Jnew[k * L.N + v]);
    }
    R Dp[3][3];
    dphi_of<R, R>(Jn, Jo, Dp);
#pragma unroll
    for (int k = 0; k < 9; k++) J[k * L.N + v] = Jn[k];
    const R j[3] = {in[1], in[2], in[3]}, B[3] = {in[11], in[12], in[13]};
    const R M2[6] = {in[4], in[5], in[6], in[7], in[8], in[9]};
    const R Cs[6] = {in[14], in[15], in[16], in[17], in[18], in[19]};
    transform_store<S, R>(L, Pout, hout, sgn, x, y, z, v, Dp, in[0], j, M2, in[10], B, Cs, literal);
}

// Chart change with interpolation, pass 1: the transformation inputs of every
// old node into mf [20][N]
template <class S, class R>
__global__ void __launch_bounds__(TPB) k_moment_fields(Lat L, const S* __restrict__ Pin, const R* __restrict__ hin,
                                                       const R* __restrict__ geo_old, R* __restrict__ mf, int literal)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= L.N) return;
    int x, y, z;
    node_coords(L, v, x, y, z);
    R in[20];
    transform_inputs<S, R>(L, Pin, hin, geo_old, x, y, z, v, literal, in);
#pragma unroll
    for (int k = 0; k < 20; k++) mf[k * L.N + v] = in[k];
}

// trilinear corners of the point p (old lattice coordinates) along one axis:
// a periodic axis wraps, a non-periodic one clamps p to [0, n - 1]
__device__ __forceinline__ void interp_axis(double p, int n, bool per, int& i0, int& i1, double& t)
{
    if (per) {
        p = fmod(p, (double)n);
        if (p < 0.0) p += n;
    } else {
        p = fmin(fmax(p, 0.0), (double)(n - 1));
    }
    const double fl = floor(p);
    i0 = (int)fl;
    t = p - fl;
    if (i0 >= n) i0 = n - 1;
    i1 = per ? (i0 + 1 == n ? 0 : i0 + 1) : (i0 + 1 < n ? i0 + 1 : n - 1);
}

// pass 2: every new node from the fields at psi(x~) = psi3[.][v]
template <class S, class R>
__global__ void __launch_bounds__(TPB) k_transform_interp(Lat L, S* __restrict__ Pout, R* __restrict__ hout,
                                                          const R* __restrict__ geo_new, const R* __restrict__ J,
                                                          const double* __restrict__ Jnew,
                                                          const double* __restrict__ psi, const R* __restrict__ mf,
                                                          int literal)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= L.N) return;
    int x, y, z;
    node_coords(L, v, x, y, z);
    int c0[3], c1[3];
    double t[3];
#pragma unroll
    for (int a = 0; a < 3; a++)
        interp_axis(psi[a * L.N + v], L.n[a], L.bclo[a] == BC_PERIODIC && L.bchi[a] == BC_PERIODIC, c0[a], c1[a],
                    t[a]);
    long long ix[8];
    double w[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int b0 = c & 1, b1 = (c >> 1) & 1, b2 = (c >> 2) & 1;
        ix[c] = nidx(L, b0 ? c1[0] : c0[0], b1 ? c1[1] : c0[1], b2 ? c1[2] : c0[2]);
        w[c] = (b0 ? t[0] : 1.0 - t[0]) * (b1 ? t[1] : 1.0 - t[1]) * (b2 ? t[2] : 1.0 - t[2]);
    }
    double Jo[9], Jn[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 8; c++) s += w[c] * double(J[k * L.N + ix[c]]);
        Jo[k] = s;
        Jn[k] = Jnew[k * L.N + v];
    }
    R Dp[3][3];
    dphi<R, R>(Jn, Jo, Dp);
    R in[20];
#pragma unroll
    for (int k = 0; k < 20; k++) {
        R s = R(0);
#pragma unroll
        for (int c = 0; c < 8; c++) s += R(w[c]) * mf[k * L.N + ix[c]];
        in[k] = s;
    }
    const R j[3] = {in[1], in[2], in[3]}, B[3] = {in[11], in[12], in[13]};
    const R M2[6] = {in[4], in[5], in[6], in[7], in[8], in[9]};
    const R Cs[6] = {in[14], in[15], in[16], in[17], in[18], in[19]};
    transform_store<S, R>(L, Pout, hout, geo_new[v], x, y, z, v, Dp, in[0], j, M2, in[10], B, Cs, literal);
}

// ---------------------------------------------------------------------------
// readout and reductions
// ---------------------------------------------------------------------------
template <class S, class R>
__global__ void __launch_bounds__(TPB) k_readout(Lat L, const S* __restrict__ P, const R* __restrict__ hist,
                                                 const R* __restrict__ geo, const R* __restrict__ J,
                                                 double* __restrict__ rho_out, double* __restrict__ u_out,
                                                 long long stride, long long v0, long long cnt, int cartesian)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    long long v = v0 + t;
    int x, y, z;
    node_coords(L, v, x, y, z);
    NodeMoments<S, R> M;
    node_moments<S, R>(L, P, hist, geo, x, y, z, v, geo[v], M);
    double u[3];
#pragma unroll
    for (int a = 0; a < 3; a++) u[a] = double(M.j[a]) / double(M.rho);
    if (rho_out) rho_out[t] = double(M.rho);
    if (u_out) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            double s = u[a];
            if (cartesian)
                s = double(J[(a * 3 + 0) * L.N + v]) * u[0] + double(J[(a * 3 + 1) * L.N + v]) * u[1] +
                    double(J[(a * 3 + 2) * L.N + v]) * u[2];
            u_out[a * stride + t] = s;
        }
    }
}

// FP64 block reduction of up to 3 values, one atomic per block and value.
template <int K>
__device__ __forceinline__ void block_reduce_add(double (&val)[K], double* acc)
{
    __shared__ double part[K][TPB / 32];
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val[k] += __shfl_down_sync(0xffffffffu, val[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) part[k][wid] = val[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = lane < (TPB / 32) ? part[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) atomicAdd(acc + k, s);
        }
    }
}

// rho of a face node (the boundary rule), out of line: few nodes take it
template <class S, class R>
__device__ __noinline__ R face_rho(const Lat& L, const S* __restrict__ P, const R* __restrict__ hist,
                                   const R* __restrict__ geo, int x, int y, int z, long long v, R sg)
{
    NodeMoments<S, R> M;
    node_moments<S, R>(L, P, hist, geo, x, y, z, v, sg, M);
    return M.rho;
}

// a value of the arithmetic's type as FP64, exactly (FP32 through the integer
// units: a conversion on the FP64 pipe costs as much as the product)
__device__ __forceinline__ double exact64(float v) { return f32_to_f64(v); }
__device__ __forceinline__ double exact64(double v) { return v; }

// Total mass: every thread sums sqrt(g) rho of the nodes v = i, i + stride, ...
// in FP64 (the product of two FP32 values is exact in FP64), then one block
// reduction; a grid of the resident blocks keeps the FP64 work per node at
// one multiply and one add.
template <class S, class R>
__global__ void __launch_bounds__(TPB, 3) k_mass(Lat L, const S* __restrict__ P, const R* __restrict__ hist,
                                              const R* __restrict__ geo, double* acc)
{
    double val[1] = {0.0};
    const unsigned N = (unsigned)L.N, n0 = L.n[0], n1 = L.n[1];
    for (unsigned v = blockIdx.x * TPB + threadIdx.x; v < N; v += gridDim.x * TPB) {
        const unsigned row = v / n0, z = row / n1;
        const int x = (int)(v - row * n0), y = (int)(row - z * n1);
        const R sg = geo[v];
        R rho;
        if (on_boundary(L, x, y, (int)z)) {
            rho = face_rho<S, R>(L, P, hist, geo, x, y, (int)z, v, sg);
        } else {
            // rho = sqrt(g)(1 + sum s) + A/2 of the pulled populations (the same sums as node_moments)
            R s[Q], m0, m1[3], m2[6];
            gather_raw<S, R>(L, P, x, y, (int)z, s);
            sums(s, m0, m1, m2);
            rho = sg * (R(1) + m0) + R(0.5) * hist[v];
        }
        val[0] += exact64(sg) * exact64(rho);
    }
    block_reduce_add<1>(val, acc);
}

template <class S, class R>
__global__ void __launch_bounds__(TPB) k_wall_force(Lat L, const S* __restrict__ P, const R* __restrict__ hist,
                                                    const R* __restrict__ geo, const R* __restrict__ J,
                                                    int axis, int side, double* acc)
{
    // one thread per node of the face
    const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
    long long nf = (long long)L.n[a1] * L.n[a2];
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double val[3] = {0.0, 0.0, 0.0};
    if (t < nf) {
        int r[3];
        r[axis] = side ? L.n[axis] - 1 : 0;
        r[a1] = (int)(t % L.n[a1]);
        r[a2] = (int)(t / L.n[a1]);
        const long long v = nidx(L, r[0], r[1], r[2]);
        Geo<R> G;
        load_metric(geo, L.N, v, G);
        NodeMoments<S, R> M;
        node_moments<S, R>(L, P, hist, geo, r[0], r[1], r[2], v, G.sg, M);
        const R ir = R(1) / M.rho, theta = R(L.theta), kv = R(L.kvisc);
        R Tn[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const int k = s6(i, axis);
            R pieq = M.rho * theta * G.gi[k] + M.j[i] * M.j[axis] * ir;
            R pi = G.sg * ((i == axis ? R(1.0 / 3.0) : R(0)) + M.m2[k]) + R(0.5) * M.Hp.C[k];
            Tn[i] = pieq + kv * (pi - pieq);
        }
        const double sgn = side ? 1.0 : -1.0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < 3; i++) s += double(J[(a * 3 + i) * L.N + v]) * double(Tn[i]);
            val[a] = sgn * s * double(G.sg);
        }
    }
    block_reduce_add<3>(val, acc);
}

template <class S, class R>
__global__ void __launch_bounds__(TPB) k_check(Lat L, const S* __restrict__ P, const R* __restrict__ hist,
                                               const R* __restrict__ geo, const R* __restrict__ J, double* acc)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double val[1] = {0.0};
    if (v < L.N) {
        int x, y, z;
        node_coords(L, v, x, y, z);
        NodeMoments<S, R> M;
        node_moments<S, R>(L, P, hist, geo, x, y, z, v, geo[v], M);
        double u[3], s2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; a++) u[a] = double(M.j[a]) / double(M.rho);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            double va = double(J[(a * 3) * L.N + v]) * u[0] + double(J[(a * 3 + 1) * L.N + v]) * u[1] +
                        double(J[(a * 3 + 2) * L.N + v]) * u[2];
            s2 += va * va;
        }
        const bool bad = !(double(M.rho) > 0.0) || !(s2 <= 0.09);  // false for NaN too
        val[0] = bad ? 1.0 : 0.0;
    }
    block_reduce_add<1>(val, acc);
}


// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <class S, class R> struct Launch {
    static S* P(const cslbm_ctx* c, int k) { return (S*)c->P[k]; }
    static R* H(const cslbm_ctx* c, int k) { return (R*)c->H[k]; }
    static R* G(const cslbm_ctx* c, int k) { return (R*)c->G[k]; }

    static void metric(const cslbm_ctx* c, const double* g6, const double* dg18, long long stride, long long v0,
                       long long cnt, int dst, int* bad)
    {
        k_metric<R><<<nblocks(cnt), TPB, 0, c->stream>>>(g6, dg18, stride, v0, cnt, G(c, dst), c->N, bad);
    }
    static void init_scatter(const cslbm_ctx* c, const double* rho, const double* u3, long long stride, long long v0,
                             long long cnt)
    {
        k_init_scatter<S, R><<<nblocks(cnt), TPB, 0, c->stream>>>(make_lat(c), rho, u3, stride, v0, cnt,
                                                                  G(c, c->gc), P(c, c->pc));
    }
    static void momentum_field(const cslbm_ctx* c)
    {
        launch_momentum<S, R>(c, make_lat(c), P(c, c->pc), H(c, c->hc), G(c, c->gc));
    }
    static int step(cslbm_ctx* c, int force_only)
    {
        Lat L = make_lat(c);
        if (force_only) {
            k_forcing<S, R><<<nblocks(c->N), TPB, 0, c->stream>>>(L, P(c, c->pc), H(c, c->hc), H(c, 1 - c->hc),
                                                                 G(c, c->gc), c->jf);
            return 1;
        }
        if constexpr (!std::is_same<R, double>::value) {
            if (c->rows.fused_ok && c->p.step_kernel == CSLBM_STEP_AUTO) {
                const int k = launch_fused_step<S>(c, L, c->pc, c->hc, c->gc, step_error_flag(c));
                if (k > 0) return k;
            }
            if (c->rows.ok) return launch_rows_step<S>(c, L, c->pc, c->hc, c->gc, step_error_flag(c));
        }
        launch_flat_step<S, R>(c, L, P(c, c->pc), P(c, 1 - c->pc), H(c, c->hc), H(c, 1 - c->hc), G(c, c->gc));
        return 2;
    }
    static void half_shift(const cslbm_ctx* c)
    {
        k_half_shift<S, R><<<nblocks(c->N), TPB, 0, c->stream>>>(make_lat(c), P(c, c->pc), H(c, c->hc), G(c, c->gc));
    }
    static void transform(const cslbm_ctx* c, const double* Jnew, long long stride, long long v0, long long cnt)
    {
        k_transform<S, R><<<nblocks(cnt), TPB, 0, c->stream>>>(make_lat(c), P(c, c->pc), P(c, 1 - c->pc), H(c, c->hc),
                                                               H(c, 1 - c->hc), G(c, c->gc), G(c, 1 - c->gc), (R*)c->J, Jnew,
                                                               stride, v0, cnt, c->p.transform_flags & 1);
    }
    static void chart_change(const cslbm_ctx* c, const double* g6, const double* dg18, const double* Jnew, int* bad)
    {
        k_chart<S, R><<<nblocks(c->N), TPB, 0, c->stream>>>(make_lat(c), P(c, c->pc), P(c, 1 - c->pc), H(c, c->hc),
                                                           H(c, 1 - c->hc), G(c, c->gc), G(c, 1 - c->gc), (R*)c->J, g6,
                                                           dg18, Jnew, c->p.transform_flags & 1, bad);
    }
    // the same with the derivatives and the Jacobian in FP32 (FP32-arithmetic
    // storage only: there they are rounded to FP32 before any use)
    static void chart_change_mixed(const cslbm_ctx* c, const double* g6, const float* dg18, const float* Jnew,
                                   int* bad)
    {
        if constexpr (!std::is_same<R, double>::value)
            k_chart<S, R, float><<<nblocks(c->N), TPB, 0, c->stream>>>(make_lat(c), P(c, c->pc), P(c, 1 - c->pc),
                                                                      H(c, c->hc), H(c, 1 - c->hc), G(c, c->gc),
                                                                      G(c, 1 - c->gc), (R*)c->J, g6, dg18, Jnew,
                                                                      c->p.transform_flags & 1, bad);
    }
    static void transform_interp(const cslbm_ctx* c, const double* Jnew, const double* psi3, void* scratch)
    {
        const int lit = c->p.transform_flags & 1;
        k_moment_fields<S, R><<<nblocks(c->N), TPB, 0, c->stream>>>(make_lat(c), P(c, c->pc), H(c, c->hc), G(c, c->gc),
                                                                   (R*)scratch, lit);
        k_transform_interp<S, R><<<nblocks(c->N), TPB, 0, c->stream>>>(make_lat(c), P(c, 1 - c->pc), H(c, 1 - c->hc),
                                                                      G(c, 1 - c->gc), (R*)c->J, Jnew, psi3,
                                                                      (const R*)scratch, lit);
    }
    static void readout(const cslbm_ctx* c, double* rho, double* u3, long long stride, long long v0, long long cnt,
                        int cartesian)
    {
        k_readout<S, R><<<nblocks(cnt), TPB, 0, c->stream>>>(make_lat(c), P(c, c->pc), H(c, c->hc), G(c, c->gc), (const R*)c->J,
                                                             rho, u3, stride, v0, cnt, cartesian);
    }
    static void mass(const cslbm_ctx* c, double* acc)
    {
        // resident blocks of TPB threads: three per SM at the kernel's register bound
        const unsigned nb = nblocks(c->N), res = 3u * (unsigned)c->n_sm;
        k_mass<S, R><<<nb < res ? nb : res, TPB, 0, c->stream>>>(make_lat(c), P(c, c->pc), H(c, c->hc), G(c, c->gc),
                                                                acc);
    }
    static void wall_force(const cslbm_ctx* c, int axis, int side, double* acc)
    {
        const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
        long long nf = (long long)c->n[a1] * c->n[a2];
        k_wall_force<S, R><<<nblocks(nf), TPB, 0, c->stream>>>(make_lat(c), P(c, c->pc), H(c, c->hc), G(c, c->gc),
                                                               (const R*)c->J, axis, side, acc);
    }
    static void check(const cslbm_ctx* c, double* acc)
    {
        k_check<S, R><<<nblocks(c->N), TPB, 0, c->stream>>>(make_lat(c), P(c, c->pc), H(c, c->hc), G(c, c->gc),
                                                            (const R*)c->J, acc);
    }
    static constexpr cslbm_ops ops()
    {
        return cslbm_ops{&metric,    &init_scatter,       &momentum_field,   &step,    &half_shift, &transform,
                         &chart_change, &chart_change_mixed, &transform_interp, &readout, &mass,       &wall_force,
                         &check};
    }
};

}  // namespace cslbm
