// Device-side building blocks of the curved-space D3Q19 lattice Boltzmann
// step (Flouris et al., arXiv 1803.07822, Sec. II and App. A/B/D).
//
// Storage convention.  The stored field is the post-collision population
// f*_l(x,t) kept at its source node x ("pull" layout): the population that
// arrives at node y at t+1 is read from y - c_l.  Reading it back gives
//     h_l(y,t+1) = f*_l(y - c_l, t) = f_l(y,t+1) - 1/2 F_l(y,t)
// (Eq. streaming), so the half-forcing of the destination is folded into the
// moments:  rho = sqrt(g) sum h + A'/2,  rho u = sqrt(g) sum h c + B'/2,
// Pi = sqrt(g) sum h c c + C'/2, with A', B', C' the forcing moments of the
// previous step.  The value stored is h - w_l (weight shift), which keeps the
// stored magnitudes small for the reduced-precision formats.
//
// The forcing history is stored as its ten Hermite coefficients (A, B^i,
// C^ij), which define F_l exactly (Eq. forcing2).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cslbm {

constexpr int Q = 19;
constexpr int NGEO = 25;   // sqrt(g), g^ij (6), Gamma^i_jk (3 x 6)
constexpr int NHIST = 10;  // A, B^i (3), C^ij (6)

// D3Q19: rest, +-x, +-y, +-z, then the twelve edge vectors (xy, xz, yz).
__host__ __device__ __forceinline__ constexpr int cvec(int l, int a)
{
    constexpr int t[Q][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                             {0, 0, 1},  {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                             {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                             {0, 1, 1},  {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
    return t[l][a];
}
// Storage plane of direction l in a population buffer [19][N]: the
// directions that share (c_y, c_z) -- and so pull from the same row -- lie
// next to each other, 0 1 2 | 3 7 10 | 4 8 9 | 5 11 14 | 6 12 13 | 15 | 16 |
// 17 | 18, so that one copy of three planes stages the rows they pull.
__host__ __device__ __forceinline__ constexpr int pslot(int l)
{
    constexpr int t[Q] = {0, 1, 2, 3, 6, 9, 12, 4, 7, 8, 5, 10, 13, 14, 11, 15, 16, 17, 18};
    return t[l];
}
// the same for a runtime l, from two words of 5-bit fields (no table in local memory)
__device__ __forceinline__ int pslot_rt(int l)
{
    const unsigned long long a = 0x515072312618820ull, b = 0x4a307adcdull;
    return (int)((l < 12 ? a >> (5 * l) : b >> (5 * (l - 12))) & 31ull);
}
// the nine staging groups: first plane, number of planes, and a direction of the group
__host__ __device__ __forceinline__ constexpr int pgroup_base(int g) { return g < 5 ? 3 * g : g + 10; }
__host__ __device__ __forceinline__ constexpr int pgroup_count(int g) { return g < 5 ? 3 : 1; }
__host__ __device__ __forceinline__ constexpr int pgroup_dir(int g) { return g == 0 ? 0 : (g < 5 ? g + 2 : g + 10); }
constexpr int PGROUPS = 9;

// Weights of the lattice quadrature: 1/3 rest, 1/18 faces, 1/36 edges.
__host__ __device__ __forceinline__ constexpr double wq(int l)
{
    return l == 0 ? 1.0 / 3.0 : (l <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
// symmetric 3x3 packed as 00,01,02,11,12,22
__host__ __device__ __forceinline__ constexpr int s6(int i, int j)
{
    return i <= j ? (i == 0 ? j : (i == 1 ? 2 + j : 5)) : (j == 0 ? i : (j == 1 ? 2 + i : 5));
}

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INFLOW = 2, BC_OUTFLOW = 3 };

// Lattice description passed by value to every kernel.
struct Lat {
    int n[3];
    int bclo[3], bchi[3];
    long long N;
    double omega;      // 1/tau
    double kvisc;      // 1 - 1/(2 tau)
    double theta;
    double fext[3];
    const double* face[6];  // contravariant boundary velocity [3][face nodes] or null
};

__host__ __device__ __forceinline__ long long nidx(const Lat& L, int x, int y, int z)
{
    return (long long)x + (long long)L.n[0] * ((long long)y + (long long)L.n[1] * z);
}

// ---------------------------------------------------------------------------
// storage conversion
// ---------------------------------------------------------------------------
template <class S> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <> struct Store<double> {
    static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------------------
// per-node geometry
// ---------------------------------------------------------------------------
template <class R> struct Geo {
    R sg, isg;     // sqrt(g), 1/sqrt(g)
    R gi[6];       // g^ij
    R gam[18];     // Gamma^i_jk at i*6 + s6(j,k)
    R gc[3];       // Gamma^j_kj (contracted), = d_k ln sqrt(g)
};

template <class R>
__device__ __forceinline__ void load_metric(const R* __restrict__ geo, long long N, long long v, Geo<R>& G)
{
    G.sg = geo[v];
    G.isg = R(1) / G.sg;
#pragma unroll
    for (int a = 0; a < 6; a++) G.gi[a] = geo[(1 + a) * N + v];
}

template <class R>
__device__ __forceinline__ void load_geo(const R* __restrict__ geo, long long N, long long v, Geo<R>& G)
{
    load_metric(geo, N, v, G);
#pragma unroll
    for (int a = 0; a < 18; a++) G.gam[a] = geo[(7 + a) * N + v];
#pragma unroll
    for (int k = 0; k < 3; k++) G.gc[k] = G.gam[0 * 6 + s6(k, 0)] + G.gam[1 * 6 + s6(k, 1)] + G.gam[2 * 6 + s6(k, 2)];
}

// ---------------------------------------------------------------------------
// Hermite recomposition (Eq. expansion-equilibrium-distribution / forcing2):
//   value_l = w_l / sqrt(g) [ b0 + b1.c / c_s^2 + b2:(c c - c_s^2 delta) / (2 c_s^4) ]
// with c_s^2 = 1/3.  b2 packed symmetric.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R hermite_l(int l, R isg, R b0, const R b1[3], const R b2[6], R trb2)
{
    const int cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
    R cc = b2[0] * (cx * cx) + b2[3] * (cy * cy) + b2[5] * (cz * cz)
         + R(2) * (b2[1] * (cx * cy) + b2[2] * (cx * cz) + b2[4] * (cy * cz));
    R v = b0 + R(3) * (b1[0] * cx + b1[1] * cy + b1[2] * cz) + R(4.5) * (cc - trb2 * R(1.0 / 3.0));
    return R(wq(l)) * isg * v;
}

// history coefficients of node v -> (A, B, b2 = C - c_s^2 delta A)
template <class R> struct Hist {
    R A, B[3], C[6];
};

template <class R>
__device__ __forceinline__ void load_hist(const R* __restrict__ h, long long N, long long v, Hist<R>& H)
{
    H.A = h[v];
#pragma unroll
    for (int a = 0; a < 3; a++) H.B[a] = h[(1 + a) * N + v];
#pragma unroll
    for (int a = 0; a < 6; a++) H.C[a] = h[(4 + a) * N + v];
}

template <class R>
__device__ __forceinline__ R forcing_l(int l, R isg, const Hist<R>& H)
{
    R b2[6];
#pragma unroll
    for (int a = 0; a < 6; a++) b2[a] = H.C[a];
    b2[0] -= H.A * R(1.0 / 3.0);
    b2[3] -= H.A * R(1.0 / 3.0);
    b2[5] -= H.A * R(1.0 / 3.0);
    return hermite_l(l, isg, H.A, H.B, b2, b2[0] + b2[3] + b2[5]);
}

// equilibrium Hermite coefficients: a0 = rho, a1 = rho u,
// a2 = rho (theta g^ij - c_s^2 delta) + rho u u   (App. B)
template <class R>
__device__ __forceinline__ void feq_coeffs(R rho, const R j[3], const R gi[6], R theta, R a2[6])
{
    R ir = R(1) / rho;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++)
            a2[s6(a, b)] = rho * theta * gi[s6(a, b)] - (a == b ? rho * R(1.0 / 3.0) : R(0)) + j[a] * j[b] * ir;
}

// ---------------------------------------------------------------------------
// gathering the populations of a node
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrapc(int v, int n)
{
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// h_l - w_l of a node whose sources y - c_l all lie inside the domain after
// periodic wrapping (true for every node that is on no non-periodic face).
template <class S, class R>
__device__ __forceinline__ void gather_raw(const Lat& L, const S* __restrict__ P, int x, int y, int z, R s[Q])
{
    // the wrapped offsets of r - c per axis, summed per population
    const unsigned n0 = L.n[0], n01 = n0 * (unsigned)L.n[1];
    unsigned ox[3], oy[3], oz[3];
#pragma unroll
    for (int c = -1; c <= 1; c++) {
        ox[c + 1] = (unsigned)wrapc(x - c, L.n[0]);
        oy[c + 1] = (unsigned)wrapc(y - c, L.n[1]) * n0;
        oz[c + 1] = (unsigned)wrapc(z - c, L.n[2]) * n01;
    }
#pragma unroll
    for (int l = 0; l < Q; l++)
        s[l] = R(Store<S>::ld(P + (long long)pslot(l) * L.N +
                              (oz[cvec(l, 2) + 1] + oy[cvec(l, 1) + 1] + ox[cvec(l, 0) + 1])));
}

// Boundary classification: rule of the highest-priority face the node lies on
// (wall > inflow > outflow; ties: lower axis, then low side), and the inner
// node = one step inward along the normal of every non-periodic face it is on.
__device__ __forceinline__ int classify(const Lat& L, const int r[3], int& axis, int& side, int in[3])
{
    int best = BC_PERIODIC, rank = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        in[a] = r[a];
        if (L.bclo[a] != BC_PERIODIC && r[a] == 0) {
            in[a] = 1;
            int rk = L.bclo[a] == BC_WALL ? 3 : (L.bclo[a] == BC_INFLOW ? 2 : 1);
            if (rk > rank) { rank = rk; best = L.bclo[a]; axis = a; side = 0; }
        }
        if (L.bchi[a] != BC_PERIODIC && r[a] == L.n[a] - 1) {
            in[a] = L.n[a] - 2;
            int rk = L.bchi[a] == BC_WALL ? 3 : (L.bchi[a] == BC_INFLOW ? 2 : 1);
            if (rk > rank) { rank = rk; best = L.bchi[a]; axis = a; side = 1; }
        }
    }
    return best;
}

__device__ __forceinline__ long long face_node(const Lat& L, int axis, const int r[3])
{
    return axis == 0 ? (long long)r[1] + (long long)L.n[1] * r[2]
         : (axis == 1 ? (long long)r[0] + (long long)L.n[0] * r[2] : (long long)r[0] + (long long)L.n[0] * r[1]);
}

// sums over the shifted populations s = h - w:
// m0 = sum s, m1 = sum s c, m2 = sum s c c (packed)
template <class R>
__device__ __forceinline__ void sums(const R s[Q], R& m0, R m1[3], R m2[6])
{
    m0 = R(0);
#pragma unroll
    for (int a = 0; a < 3; a++) m1[a] = R(0);
#pragma unroll
    for (int a = 0; a < 6; a++) m2[a] = R(0);
#pragma unroll
    for (int l = 0; l < Q; l++) {
        const int cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
        m0 += s[l];
        if (cx) m1[0] += cx * s[l];
        if (cy) m1[1] += cy * s[l];
        if (cz) m1[2] += cz * s[l];
        if (cx) m2[0] += s[l];
        if (cy) m2[3] += s[l];
        if (cz) m2[5] += s[l];
        if (cx * cy) m2[1] += (cx * cy) * s[l];
        if (cx * cz) m2[2] += (cx * cz) * s[l];
        if (cy * cz) m2[4] += (cy * cz) * s[l];
    }
}

// Is the node on a non-periodic face?
__device__ __forceinline__ bool on_boundary(const Lat& L, int x, int y, int z)
{
    return (L.bclo[0] != BC_PERIODIC && (x == 0 || x == L.n[0] - 1)) ||
           (L.bclo[1] != BC_PERIODIC && (y == 0 || y == L.n[1] - 1)) ||
           (L.bclo[2] != BC_PERIODIC && (z == 0 || z == L.n[2] - 1));
}

// The boundary rule (reading of Sec. IV.A / VI.A: nodes on the wall) from
// the inner node's pulled populations si = h - w, metric Gi and history Hi:
// non-equilibrium extrapolation for wall and inflow nodes (velocity uw,
// contravariant), zero-gradient copy for outflow nodes, both scaled by
// sqrt(g_inner) / sqrt(g_node); returns the node's s = h - w with h = f -
// F'/2 from its own history Hw and metric Gw.
template <class R>
__device__ __forceinline__ void boundary_rule(const Lat& L, int bc, const R si[Q], const Geo<R>& Gi, const Hist<R>& Hi,
                                              const Geo<R>& Gw, const Hist<R>& Hw, const R uw[3], R s[Q])
{
    // Written out, the rule is
    //   outflow:       s_l = ratio f_l(i) - F_l(w)/2 - w_l,
    //   wall, inflow:  s_l = feq_l(rho_i, rho_i u_w; w) + ratio (f_l(i) - feq_l(rho_i, j_i; i))
    //                        - F_l(w)/2 - w_l,
    // with f_l(i) = si_l + w_l + F_l(i)/2 and ratio = sqrt(g_i) / sqrt(g_w).  Every
    // feq_l and F_l is w_l / sqrt(g) P_l(b0, b1, b2) of its node, P_l(b) = b0 + 3 b1.c
    // + 4.5 (b2 : c c - tr b2 / 3) linear in b, and ratio / sqrt(g_i) = 1 / sqrt(g_w),
    // so the terms combine into one expansion:
    //   s_l = ratio si_l + (ratio - 1) w_l + w_l / sqrt(g_w) P_l(E),
    //   E = ((A, B, b2)_i - (A, B, b2)_w) / 2   (b2 = C - c_s^2 delta A of the histories)
    //     + (0, j_w - j_i, a2eq_w - a2eq_i)     (wall and inflow nodes only; rho cancels).
    const R ratio = Gi.sg * Gw.isg;
    const R e0 = R(0.5) * (Hi.A - Hw.A);
    R e1[3], e2[6];
#pragma unroll
    for (int a = 0; a < 3; a++) e1[a] = R(0.5) * (Hi.B[a] - Hw.B[a]);
#pragma unroll
    for (int k = 0; k < 6; k++) e2[k] = R(0.5) * (Hi.C[k] - Hw.C[k]) - ((k == 0 || k == 3 || k == 5) ? e0 * R(1.0 / 3.0) : R(0));
    if (bc != BC_OUTFLOW) {
        R m0, m1[3], m2[6];
        sums(si, m0, m1, m2);
        const R rho = Gi.sg * (R(1) + m0) + R(0.5) * Hi.A;
        R j[3], jw[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            j[a] = Gi.sg * m1[a] + R(0.5) * Hi.B[a];
            jw[a] = rho * uw[a];
        }
        R a2w[6], a2i[6];
        feq_coeffs(rho, jw, Gw.gi, R(L.theta), a2w);
        feq_coeffs(rho, j, Gi.gi, R(L.theta), a2i);
#pragma unroll
        for (int a = 0; a < 3; a++) e1[a] += jw[a] - j[a];
#pragma unroll
        for (int k = 0; k < 6; k++) e2[k] += a2w[k] - a2i[k];
    }
    const R tr = e2[0] + e2[3] + e2[5];
#pragma unroll
    for (int l = 0; l < Q; l++) s[l] = ratio * si[l] + (ratio - R(1)) * R(wq(l)) + hermite_l(l, Gw.isg, e0, e1, e2, tr);
}

// the imposed velocity of face (axis, side) at node r (zero without one)
template <class R>
__device__ __forceinline__ void face_velocity(const Lat& L, int axis, int side, const int r[3], R uw[3])
{
    uw[0] = uw[1] = uw[2] = R(0);
    const double* fv = L.face[axis * 2 + side];
    if (fv) {
        long long fn = face_node(L, axis, r);
        long long nf = axis == 0 ? (long long)L.n[1] * L.n[2] : (axis == 1 ? (long long)L.n[0] * L.n[2] : (long long)L.n[0] * L.n[1]);
#pragma unroll
        for (int a = 0; a < 3; a++) uw[a] = R(fv[a * nf + fn]);
    }
}

// Populations s = h - w of a boundary node from the boundary rule applied to
// its inner node (boundary_rule), everything gathered from global memory.
// Kept out of line where it matters (see boundary_site): it runs for the few
// nodes on the faces.
// (the node's own metric and history Gw, Hw supplied by the caller)
template <class S, class R>
__device__ __forceinline__ void boundary_pops_w(const Lat& L, const S* __restrict__ P, const R* __restrict__ hist,
                                                const R* __restrict__ geo, int x, int y, int z, const Geo<R>& Gw,
                                                const Hist<R>& Hw, R s[Q])
{
    int r[3] = {x, y, z}, in[3], axis = 0, side = 0;
    const int bc = classify(L, r, axis, side, in);
    const long long N = L.N;
    const long long vi = nidx(L, in[0], in[1], in[2]);
    R si[Q];
    gather_raw<S, R>(L, P, in[0], in[1], in[2], si);
    Geo<R> Gi;
    load_metric(geo, N, vi, Gi);
    Hist<R> Hi;
    load_hist(hist, N, vi, Hi);
    R uw[3];
    face_velocity(L, axis, side, r, uw);
    boundary_rule(L, bc, si, Gi, Hi, Gw, Hw, uw, s);
}
template <class S, class R>
__device__ __forceinline__ void boundary_pops(const Lat& L, const S* __restrict__ P, const R* __restrict__ hist,
                                           const R* __restrict__ geo, int x, int y, int z, R s[Q])
{
    const long long N = L.N, vw = nidx(L, x, y, z);
    Geo<R> Gw;
    load_metric(geo, N, vw, Gw);
    Hist<R> Hw;
    load_hist(hist, N, vw, Hw);
    boundary_pops_w<S, R>(L, P, hist, geo, x, y, z, Gw, Hw, s);
}

// Node state: shifted populations s = h - w of any node (boundary nodes
// through the boundary rule).
template <class S, class R>
__device__ __forceinline__ void node_pops(const Lat& L, const S* __restrict__ P, const R* __restrict__ hist,
                                          const R* __restrict__ geo, int x, int y, int z, R s[Q])
{
    if (on_boundary(L, x, y, z)) boundary_pops<S, R>(L, P, hist, geo, x, y, z, s);
    else gather_raw<S, R>(L, P, x, y, z, s);
}

// ---------------------------------------------------------------------------
// forcing moments (Eqs. forcing-A/B/C), in terms of the contracted symbol
// Gamma^j_kj =: gc_k (Gamma is symmetric in its lower indices):
//   A    = -2 gc_i j^i
//   B^i  = F_ext^i - 2 gc_j T^ij - Gamma^i_jk T^jk
//   C^ij = c_s^2 (dbar_j j^i + dbar_i j^j + delta^ij dbar_k j^k)
//        - theta (g^jk nabla_k j^i + g^ik nabla_k j^j + g^ij nabla_k j^k)
// with dbar_k j^i = D_k j^i - gc_k j^i, nabla_k j^i = D_k j^i + Gamma^i_kl j^l,
// D[k][i] the lattice gradient d_k (rho u^i).
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void forcing_moments(const Lat& L, const Geo<R>& G, const R j[3], const R T[6],
                                                const R D[3][3], Hist<R>& out)
{
    const R theta = R(L.theta);
    out.A = R(-2) * (G.gc[0] * j[0] + G.gc[1] * j[1] + G.gc[2] * j[2]);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        R b = R(L.fext[i]);
#pragma unroll
        for (int jj = 0; jj < 3; jj++) b -= R(2) * G.gc[jj] * T[s6(i, jj)];
#pragma unroll
        for (int jj = 0; jj < 3; jj++)
#pragma unroll
            for (int k = 0; k < 3; k++) b -= G.gam[i * 6 + s6(jj, k)] * T[s6(jj, k)];
        out.B[i] = b;
    }
    R bard[3][3], cov[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int i = 0; i < 3; i++) {
            bard[k][i] = D[k][i] - G.gc[k] * j[i];
            R s = D[k][i];
#pragma unroll
            for (int l = 0; l < 3; l++) s += G.gam[i * 6 + s6(k, l)] * j[l];
            cov[k][i] = s;
        }
    const R divbar = bard[0][0] + bard[1][1] + bard[2][2];
    const R divcov = cov[0][0] + cov[1][1] + cov[2][2];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int jj = i; jj < 3; jj++) {
            R c = R(1.0 / 3.0) * (bard[jj][i] + bard[i][jj] + (i == jj ? divbar : R(0)));
            R t = G.gi[s6(i, jj)] * divcov;
#pragma unroll
            for (int k = 0; k < 3; k++) t += G.gi[s6(jj, k)] * cov[k][i] + G.gi[s6(i, k)] * cov[k][jj];
            out.C[s6(i, jj)] = c - theta * t;
        }
}

}  // namespace cslbm
