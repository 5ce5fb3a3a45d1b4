// Adjoint of the LBM step for gradients of a wall force with respect to the
// geometry (FP32 or FP64 storage, walls at rest and periodic faces).
//
// One backward step takes the adjoint of the state at time t+1 (populations
// and history, "lambda") to time t, given the forward state at time t in the
// context, and adds the step's contribution to the adjoint of the geometry.
// The step's dependencies are local except three, each handled by a pass of
// its own:
//   A  (every node) the forward step of the node recomputed and reversed
//      (adj::step_reverse): adjoints of its pulled populations (field lS),
//      of its history at t (lH at t), of its geometry (lGeo, accumulated)
//      and of its lattice gradient D (field lD).  A face node reverses the
//      ghost extrapolation of its stencil and adds the rho-u adjoint of the
//      real sites to lJF with atomics;
//   B  (every node y) the rho-u adjoint of y gathered from the lD of the
//      interior nodes whose stencil holds y, plus lJF; since
//      j(y) = sqrt(g) sum_l s_l c_l + B(y)/2 it goes to lS(y), to sqrt(g)
//      and to the history B of y;
//   C  (face nodes) the boundary rule reversed: lS of the face node goes to
//      the pulled populations of its inner node, both nodes' metric and
//      history (atomics: edge and corner nodes share inner nodes);
//   D  (every slot) the pull reversed: the adjoint of stored value (l, y) is
//      lS_l of the node that pulls it, y + c_l, or zero when that node is a
//      face node (the boundary rule ignores its pulled values).
// A pass's forward quantities come from the context's state at time t and
// from rho u at time t, which the backward step recomputes first.
#include <cstdio>
#include <string>

#include "ctx.h"
#include "make_lat.h"
#include "adjoint.cuh"

namespace cslbm {
namespace adj {

constexpr int TB_A = 128;

template <class R> struct Bufs {
    R* lP[2];   // [19][N] adjoint of the stored populations (current: lp)
    R* lH[2];   // [10][N] adjoint of the history
    R* lS;      // [19][N] adjoint of each node's pulled (face node: rule) populations
    R* lD;      // [9][N]  adjoint of each node's lattice gradient D[k][i] at k*3+i
    R* lJF;     // [3][N]  rho-u adjoint scattered by face nodes
    R* lGeo;    // [25][N] adjoint of the geometry, summed over the steps
    double* lJ; // [9][N]  adjoint of the chart Jacobian (wall force)
};

template <class R> __device__ __forceinline__ void add(R* p, R v) { atomicAdd(p, v); }

// (32-bit arithmetic: a context holds fewer than 2^32 nodes)
__device__ __forceinline__ void node_xyz(const Lat& L, long long v, int& x, int& y, int& z)
{
    const unsigned vu = (unsigned)v, n0 = L.n[0], n1 = L.n[1], row = vu / n0, zr = row / n1;
    x = (int)(vu - row * n0);
    y = (int)(row - zr * n1);
    z = (int)zr;
}

// ghost extrapolation of a stencil site reversed: the adjoint lj of the
// site's rho u distributed onto the real nodes it was built from
template <class R>
__device__ __noinline__ void site_reverse(const Lat& L, int x, int y, int z, R lj0, R lj1, R lj2, R* lJF)
{
    const R lj[3] = {lj0, lj1, lj2};
    int x0, x1, y0, y1, z0, z1;
    float wx0, wx1, wy0, wy1, wz0, wz1;
    site_axis(x, L.n[0], L.bclo[0] == BC_PERIODIC, L.bchi[0] == BC_PERIODIC, x0, x1, wx0, wx1);
    site_axis(y, L.n[1], L.bclo[1] == BC_PERIODIC, L.bchi[1] == BC_PERIODIC, y0, y1, wy0, wy1);
    site_axis(z, L.n[2], L.bclo[2] == BC_PERIODIC, L.bchi[2] == BC_PERIODIC, z0, z1, wz0, wz1);
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 2; k++)
            for (int m = 0; m < 2; m++) {
                const float w = (i ? wx1 : wx0) * (k ? wy1 : wy0) * (m ? wz1 : wz0);
                if (w == 0.0f) continue;
                const long long v = nidx(L, i ? x1 : x0, k ? y1 : y0, m ? z1 : z0);
#pragma unroll
                for (int a = 0; a < 3; a++) add(lJF + a * L.N + v, R(w) * lj[a]);
            }
}

// the forward inputs of a face node (boundary rule, ghost stencil), out of
// line so that the interior path keeps its registers
template <class R>
__device__ __noinline__ void face_inputs(const Lat& L, const R* __restrict__ P, const R* __restrict__ H,
                                         const R* __restrict__ geo, const Mom4<R>* __restrict__ jf, int x, int y,
                                         int z, R* s, R* d)
{
    boundary_pops<R, R>(L, P, H, geo, x, y, z, s);
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const int l = 2 * k + 1, cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
        const Mom4<R> p = mom_site(L, jf, x + cx, y + cy, z + cz), m = mom_site(L, jf, x - cx, y - cy, z - cz);
        d[3 * k + 0] = p.x - m.x;
        d[3 * k + 1] = p.y - m.y;
        d[3 * k + 2] = p.z - m.z;
    }
}

// pass A
template <class R>
__global__ void __launch_bounds__(TB_A, 4) k_adj_local(Lat L, const R* __restrict__ P, const R* __restrict__ H,
                                                     const R* __restrict__ geo, const Mom4<R>* __restrict__ jf,
                                                     const R* __restrict__ lPo, const R* __restrict__ lHo,
                                                     Bufs<R> B, R* __restrict__ lHi)
{
    // 32-bit node arithmetic (a context holds fewer than 2^32 nodes)
    const unsigned vu = blockIdx.x * TB_A + threadIdx.x;
    if (vu >= (unsigned)L.N) return;
    const long long v = vu, N = L.N;
    const unsigned n0 = L.n[0], n1 = L.n[1], row = vu / n0, zr = row / n1;
    const int x = (int)(vu - row * n0), y = (int)(row - zr * n1), z = (int)zr;
    const bool face = on_boundary(L, x, y, z);
    R s[Q];
    R d[9][3];
    if (face) {
        R sf[Q], df[27];
        face_inputs<R>(L, P, H, geo, jf, x, y, z, sf, df);
#pragma unroll
        for (int l = 0; l < Q; l++) s[l] = sf[l];
#pragma unroll
        for (int k = 0; k < 9; k++)
#pragma unroll
            for (int i = 0; i < 3; i++) d[k][i] = df[3 * k + i];
    } else {
        gather_raw<R, R>(L, P, x, y, z, s);
        const Nbr nb = nbr_index(L, x, y, z, +1);  // sites x + c, wrapped
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const int l = 2 * k + 1, cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
            const Mom4<R> p = jf[nbr_off(nb, cx, cy, cz)], m = jf[nbr_off(nb, -cx, -cy, -cz)];
            d[k][0] = p.x - m.x;
            d[k][1] = p.y - m.y;
            d[k][2] = p.z - m.z;
        }
    }
    GeoT<R> G;
    HistT<R> Hp;
    load_geo_hist(geo, H, (unsigned)v, (unsigned)N, G, Hp);
    R lout[Q];
#pragma unroll
    for (int l = 0; l < Q; l++) lout[l] = lPo[l * N + v];
    HistT<R> lH, lHp;
    lH.A = lHo[v];
    lHp.A = R(0);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lH.B[a] = lHo[(1 + a) * N + v];
        lHp.B[a] = R(0);
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
        lH.C[k] = lHo[(4 + k) * N + v];
        lHp.C[k] = R(0);
    }
    R ls[Q], lgeo[NG], lD[3][3];
#pragma unroll
    for (int l = 0; l < Q; l++) ls[l] = R(0);
#pragma unroll
    for (int k = 0; k < NG; k++) lgeo[k] = R(0);
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int i = 0; i < 3; i++) lD[k][i] = R(0);
    step_reverse(L, s, G, Hp, d, lout, lH, ls, lHp, lgeo, lD);
#pragma unroll
    for (int l = 0; l < Q; l++) B.lS[l * N + v] = ls[l];
    lHi[v] = lHp.A;
#pragma unroll
    for (int a = 0; a < 3; a++) lHi[(1 + a) * N + v] = lHp.B[a];
#pragma unroll
    for (int k = 0; k < 6; k++) lHi[(4 + k) * N + v] = lHp.C[k];
#pragma unroll
    for (int k = 0; k < NG; k++) B.lGeo[k * N + v] += lgeo[k];
    if (face) {
        R ld[9][3];
        gradient_reverse(lD, ld);
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const int l = 2 * k + 1, cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
            site_reverse(L, x + cx, y + cy, z + cz, ld[k][0], ld[k][1], ld[k][2], B.lJF);
            site_reverse(L, x - cx, y - cy, z - cz, -ld[k][0], -ld[k][1], -ld[k][2], B.lJF);
        }
#pragma unroll
        for (int q = 0; q < 9; q++) B.lD[q * N + v] = R(0);
    } else {
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int i = 0; i < 3; i++) B.lD[(k * 3 + i) * N + v] = lD[k][i];
    }
}

// pass B
template <class R>
__global__ void __launch_bounds__(256) k_adj_gather(Lat L, const R* __restrict__ H, const R* __restrict__ geo,
                                                     const Mom4<R>* __restrict__ jf, Bufs<R> B, R* __restrict__ lHi)
{
    const long long v = blockIdx.x * 256LL + threadIdx.x;
    if (v >= L.N) return;
    const long long N = L.N;
    int x, y, z;
    node_xyz(L, v, x, y, z);
    R lj[3] = {B.lJF[v], B.lJF[N + v], B.lJF[2 * N + v]};
    // interior nodes x' = y - c whose stencil site x' + c is this node
#pragma unroll
    for (int l = 1; l < Q; l++) {
        const int cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
        int r[3] = {x - cx, y - cy, z - cz};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (r[a] < 0 || r[a] >= L.n[a]) {
                if ((r[a] < 0 ? L.bclo[a] : L.bchi[a]) == BC_PERIODIC) r[a] = wrapc(r[a], L.n[a]);
                else ok = false;
            }
        if (!ok || on_boundary(L, r[0], r[1], r[2])) continue;
        const long long u = nidx(L, r[0], r[1], r[2]);
        const R w = R(3.0 * wq(l));
        const int c[3] = {cx, cy, cz};
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (!c[k]) continue;
#pragma unroll
            for (int i = 0; i < 3; i++) lj[i] += w * R(c[k]) * B.lD[(k * 3 + i) * N + u];
        }
    }
    // j(y) = sqrt(g) m1 + B/2 with m1 = (j - B/2) / sqrt(g)
    const R sg = geo[v];
    const Mom4<R> jv = jf[v];
    const R jj[3] = {jv.x, jv.y, jv.z};
    R lsg = R(0);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const R Bh = H[(1 + a) * N + v];
        lsg += (jj[a] - R(0.5) * Bh) / sg * lj[a];
        lHi[(1 + a) * N + v] += R(0.5) * lj[a];
    }
    B.lGeo[v] += lsg;
#pragma unroll
    for (int l = 0; l < Q; l++) {
        R t = R(0);
#pragma unroll
        for (int a = 0; a < 3; a++) t += R(cvec(l, a)) * lj[a];
        B.lS[l * N + v] += sg * t;
    }
}

// pass C: the boundary rule reversed, one thread per face node
template <class R>
__global__ void __launch_bounds__(128) k_adj_boundary(const __grid_constant__ Lat L, const __grid_constant__ FaceList f,
                                                       const R* __restrict__ P, const R* __restrict__ H,
                                                       const R* __restrict__ geo, Bufs<R> B, R* __restrict__ lHi)
{
    const long long t = blockIdx.x * 128LL + threadIdx.x;
    if (t >= f.start[f.nseg]) return;
    int lo0 = 0, lo1 = 0, lo2 = 0, len0 = 1, len1 = 1;
    long long st = 0;
#pragma unroll
    for (int k = 0; k < 6; k++)
        if (k < f.nseg && t >= f.start[k]) {
            lo0 = f.lo[k][0];
            lo1 = f.lo[k][1];
            lo2 = f.lo[k][2];
            len0 = f.len[k][0];
            len1 = f.len[k][1];
            st = f.start[k];
        }
    const long long r = t - st, q = r / len0;
    int w[3] = {lo0 + (int)(r - q * len0), lo1 + (int)(q % len1), lo2 + (int)(q / len1)};
    int in[3], axis = 0, side = 0;
    const int bc = classify(L, w, axis, side, in);
    const long long N = L.N, vw = nidx(L, w[0], w[1], w[2]), vi = nidx(L, in[0], in[1], in[2]);
    R si[Q];
    gather_raw<R, R>(L, P, in[0], in[1], in[2], si);
    Geo<R> Gi, Gw;
    load_metric(geo, N, vi, Gi);
    load_metric(geo, N, vw, Gw);
    Hist<R> Hi, Hw;
    load_hist(H, N, vi, Hi);
    load_hist(H, N, vw, Hw);
    R uw[3] = {R(0), R(0), R(0)};
    const double* fv = nullptr;
#pragma unroll
    for (int k = 0; k < 6; k++)
        if (k == axis * 2 + side) fv = L.face[k];
    if (fv) {
        const long long fn = face_node(L, axis, w);
        const long long nf = axis == 0 ? (long long)L.n[1] * L.n[2]
                                       : (axis == 1 ? (long long)L.n[0] * L.n[2] : (long long)L.n[0] * L.n[1]);
#pragma unroll
        for (int a = 0; a < 3; a++) uw[a] = R(fv[a * nf + fn]);
    }
    R ls[Q], lsi[Q], lgi_i[7], lgi_w[7];
#pragma unroll
    for (int l = 0; l < Q; l++) {
        ls[l] = B.lS[l * N + vw];
        lsi[l] = R(0);
    }
#pragma unroll
    for (int k = 0; k < 7; k++) lgi_i[k] = lgi_w[k] = R(0);
    Hist<R> lHi_, lHw_;
    lHi_.A = lHw_.A = R(0);
#pragma unroll
    for (int a = 0; a < 3; a++) lHi_.B[a] = lHw_.B[a] = R(0);
#pragma unroll
    for (int k = 0; k < 6; k++) lHi_.C[k] = lHw_.C[k] = R(0);
    boundary_reverse(L, bc, si, Gi, Gw, Hi, Hw, uw, ls, lsi, lgi_i, lgi_w, lHi_, lHw_);
#pragma unroll
    for (int l = 0; l < Q; l++) add(B.lS + l * N + vi, lsi[l]);
#pragma unroll
    for (int k = 0; k < 7; k++) {
        add(B.lGeo + k * N + vi, lgi_i[k]);
        add(B.lGeo + k * N + vw, lgi_w[k]);
    }
    add(lHi + vi, lHi_.A);
    add(lHi + vw, lHw_.A);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        add(lHi + (1 + a) * N + vi, lHi_.B[a]);
        add(lHi + (1 + a) * N + vw, lHw_.B[a]);
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
        add(lHi + (4 + k) * N + vi, lHi_.C[k]);
        add(lHi + (4 + k) * N + vw, lHw_.C[k]);
    }
}

// pass D: the pull reversed
template <class R>
__global__ void __launch_bounds__(256) k_adj_pull(Lat L, const R* __restrict__ lS, R* __restrict__ lPi)
{
    const long long v = blockIdx.x * 256LL + threadIdx.x;
    if (v >= L.N) return;
    int x, y, z;
    node_xyz(L, v, x, y, z);
#pragma unroll
    for (int l = 0; l < Q; l++) {
        int r[3] = {x + cvec(l, 0), y + cvec(l, 1), z + cvec(l, 2)};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (r[a] < 0 || r[a] >= L.n[a]) {
                if ((r[a] < 0 ? L.bclo[a] : L.bchi[a]) == BC_PERIODIC) r[a] = wrapc(r[a], L.n[a]);
                else ok = false;
            }
        R val = R(0);
        if (ok && !on_boundary(L, r[0], r[1], r[2])) val = lS[l * L.N + nidx(L, r[0], r[1], r[2])];
        lPi[l * L.N + v] = val;
    }
}

// seed: the adjoint of e . F (F the force of the fluid on face (axis, side),
// k_wall_force) onto the face nodes' populations (lS, before the boundary
// rule), history, geometry and chart Jacobian
template <class R>
__global__ void __launch_bounds__(128) k_adj_seed_force(Lat L, const R* __restrict__ P, const R* __restrict__ H,
                                                         const R* __restrict__ geo, const R* __restrict__ J,
                                                         int axis, int side, double e0, double e1, double e2,
                                                         Bufs<R> B, R* __restrict__ lHo)
{
    const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
    const long long nf = (long long)L.n[a1] * L.n[a2];
    const long long t = blockIdx.x * 128LL + threadIdx.x;
    if (t >= nf) return;
    int r[3];
    r[axis] = side ? L.n[axis] - 1 : 0;
    r[a1] = (int)(t % L.n[a1]);
    r[a2] = (int)(t / L.n[a1]);
    const long long N = L.N, v = nidx(L, r[0], r[1], r[2]);
    R s[Q];
    node_pops<R, R>(L, P, H, geo, r[0], r[1], r[2], s);
    Geo<R> G;
    load_metric(geo, N, v, G);
    Hist<R> Hp;
    load_hist(H, N, v, Hp);
    Moms<R> M;
    moments_of(s, M);
    const R th = R(L.theta), kv = R(L.kvisc), sg = G.sg;
    const R rho = sg * (R(1) + M.m0) + R(0.5) * Hp.A, ir = R(1) / rho;
    R j[3];
#pragma unroll
    for (int a = 0; a < 3; a++) j[a] = sg * M.m1[a] + R(0.5) * Hp.B[a];
    R Tn[3];
    int kk[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int k = s6(i, axis);
        kk[i] = k;
        const R pieq = rho * th * G.gi[k] + j[i] * j[axis] * ir;
        const R pi = sg * ((i == axis ? R(1.0 / 3.0) : R(0)) + M.m2[k]) + R(0.5) * Hp.C[k];
        Tn[i] = pieq + kv * (pi - pieq);
    }
    const double sgn = side ? 1.0 : -1.0, e[3] = {e0, e1, e2};
    R lTn[3];
    double lsg = 0.0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double a = 0.0;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            a += e[b] * double(J[(b * 3 + i) * N + v]);
            B.lJ[(b * 3 + i) * N + v] += sgn * double(sg) * e[b] * double(Tn[i]);
        }
        lTn[i] = R(sgn * double(sg) * a);
        lsg += sgn * a * double(Tn[i]);
    }
    R lsgR = R(lsg), lrho = R(0), lir = R(0), lj[3] = {0, 0, 0}, lm0 = R(0), lm1[3] = {0, 0, 0},
      lm2[6] = {0, 0, 0, 0, 0, 0}, lgi[6] = {0, 0, 0, 0, 0, 0}, lA = R(0), lBv[3] = {0, 0, 0}, lC[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int k = kk[i];
        const R lpi = kv * lTn[i], lpe = (R(1) - kv) * lTn[i];
        lsgR += lpi * ((i == axis ? R(1.0 / 3.0) : R(0)) + M.m2[k]);
        lm2[k] += lpi * sg;
        lC[k] += R(0.5) * lpi;
        lrho += lpe * th * G.gi[k];
        lgi[k] += lpe * rho * th;
        lj[i] += lpe * j[axis] * ir;
        lj[axis] += lpe * j[i] * ir;
        lir += lpe * j[i] * j[axis];
    }
    lrho -= ir * ir * lir;
    lsgR += (R(1) + M.m0) * lrho;
    lm0 += sg * lrho;
    lA += R(0.5) * lrho;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lsgR += M.m1[a] * lj[a];
        lm1[a] += sg * lj[a];
        lBv[a] += R(0.5) * lj[a];
    }
    R ls[Q];
#pragma unroll
    for (int l = 0; l < Q; l++) ls[l] = R(0);
    moments_reverse(lm0, lm1, lm2, ls);
#pragma unroll
    for (int l = 0; l < Q; l++) B.lS[l * N + v] += ls[l];
    B.lGeo[v] += lsgR;
#pragma unroll
    for (int k = 0; k < 6; k++) B.lGeo[(1 + k) * N + v] += lgi[k];
    lHo[v] += lA;
#pragma unroll
    for (int a = 0; a < 3; a++) lHo[(1 + a) * N + v] += lBv[a];
#pragma unroll
    for (int k = 0; k < 6; k++) lHo[(4 + k) * N + v] += lC[k];
}

// the rest initialisation reversed, every node
template <class R>
__global__ void __launch_bounds__(256) k_adj_init(Lat L, const R* __restrict__ geo, const R* __restrict__ lP,
                                                   const R* __restrict__ lH, R* __restrict__ lGeo)
{
    const long long v = blockIdx.x * 256LL + threadIdx.x;
    if (v >= L.N) return;
    const long long N = L.N;
    int x, y, z;
    node_xyz(L, v, x, y, z);
    R ls0[Q];
#pragma unroll
    for (int l = 0; l < Q; l++) {
        int r[3] = {x - cvec(l, 0), y - cvec(l, 1), z - cvec(l, 2)};
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (r[a] < 0 || r[a] >= L.n[a]) {
                if ((r[a] < 0 ? L.bclo[a] : L.bchi[a]) == BC_PERIODIC) r[a] = wrapc(r[a], L.n[a]);
                else ok = false;
            }
        ls0[l] = ok ? lP[l * N + nidx(L, r[0], r[1], r[2])] : R(0);
    }
    GeoT<R> G;
    HistT<R> dummy;
    load_geo_hist(geo, lH, (unsigned)v, (unsigned)N, G, dummy);
    const R lB0[3] = {lH[N + v], lH[2 * N + v], lH[3 * N + v]};
    R lgeo[NG];
#pragma unroll
    for (int k = 0; k < NG; k++) lgeo[k] = R(0);
    init_reverse(L, G, ls0, lB0, lgeo);
#pragma unroll
    for (int k = 0; k < NG; k++) lGeo[k * N + v] += lgeo[k];
}

// the metric kernel reversed (FP64), every node
template <class R>
__global__ void __launch_bounds__(128) k_adj_metric(long long N, const double* __restrict__ g6,
                                                     const double* __restrict__ dg18, const R* __restrict__ lGeo,
                                                     double* __restrict__ lg6, double* __restrict__ ldg18)
{
    const long long v = blockIdx.x * 128LL + threadIdx.x;
    if (v >= N) return;
    double g[6], dg[3][6], lgeo[NG], lg[6], ldg[3][6];
#pragma unroll
    for (int k = 0; k < 6; k++) g[k] = g6[k * N + v];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int k = 0; k < 6; k++) dg[a][k] = dg18[(a * 6 + k) * N + v];
#pragma unroll
    for (int k = 0; k < NG; k++) lgeo[k] = double(lGeo[k * N + v]);
    metric_reverse(g, dg, lgeo, lg, ldg);
#pragma unroll
    for (int k = 0; k < 6; k++) lg6[k * N + v] = lg[k];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int k = 0; k < 6; k++) ldg18[(a * 6 + k) * N + v] = ldg[a][k];
}

template <class R> Bufs<R> bufs(const cslbm_ctx* c)
{
    const size_t N = c->N;
    char* p = (char*)c->adj.ws;
    Bufs<R> B;
    size_t o = 0;
    auto take = [&](size_t n) {
        void* q = p + o;
        o += (n + 63) / 64 * 64;
        return q;
    };
    for (int k = 0; k < 2; k++) B.lP[k] = (R*)take(19 * N * sizeof(R));
    for (int k = 0; k < 2; k++) B.lH[k] = (R*)take(10 * N * sizeof(R));
    B.lS = (R*)take(19 * N * sizeof(R));
    B.lD = (R*)take(9 * N * sizeof(R));
    B.lJF = (R*)take(3 * N * sizeof(R));
    B.lGeo = (R*)take(25 * N * sizeof(R));
    B.lJ = (double*)take(9 * N * sizeof(double));
    return B;
}
inline size_t adj_bytes(const cslbm_ctx* c)
{
    const size_t N = c->N, r = c->r_bytes;
    auto a = [](size_t n) { return (n + 63) / 64 * 64; };
    return 2 * a(19 * N * r) + 2 * a(10 * N * r) + a(19 * N * r) + a(9 * N * r) + a(3 * N * r) + a(25 * N * r) +
           a(9 * N * 8);
}

unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// the boundary rule and pull reversed: lS -> lP[dst], history adjoint in lH[dst]
template <class R> void finish_step(cslbm_ctx* c, const Lat& L, Bufs<R>& B, int dst)
{
    const FaceList f = face_list(c);
    const long long nfc = f.start[f.nseg];
    if (nfc > 0)
        k_adj_boundary<R><<<nb(nfc, 128), 128, 0, c->stream>>>(L, f, (const R*)c->P[c->pc], (const R*)c->H[c->hc],
                                                               (const R*)c->G[c->gc], B, B.lH[dst]);
    k_adj_pull<R><<<nb(c->N, 256), 256, 0, c->stream>>>(L, B.lS, B.lP[dst]);
}

template <class R> void seed(cslbm_ctx* c, int axis, int side, const double e[3])
{
    Lat L = make_lat(c);
    Bufs<R> B = bufs<R>(c);
    const int lp = c->adj.lp;
    const size_t N = c->N;
    cudaMemsetAsync(B.lS, 0, 19 * N * sizeof(R), c->stream);
    cudaMemsetAsync(B.lH[lp], 0, 10 * N * sizeof(R), c->stream);
    cudaMemsetAsync(B.lGeo, 0, 25 * N * sizeof(R), c->stream);
    cudaMemsetAsync(B.lJ, 0, 9 * N * sizeof(double), c->stream);
    const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
    const long long nf = (long long)c->n[a1] * c->n[a2];
    k_adj_seed_force<R><<<nb(nf, 128), 128, 0, c->stream>>>(L, (const R*)c->P[c->pc], (const R*)c->H[c->hc],
                                                            (const R*)c->G[c->gc], (const R*)c->J, axis, side, e[0], e[1], e[2],
                                                            B, B.lH[lp]);
    finish_step<R>(c, L, B, lp);
}

template <class R> void backward(cslbm_ctx* c)
{
    Lat L = make_lat(c);
    Bufs<R> B = bufs<R>(c);
    const int lp = c->adj.lp, dst = 1 - lp;
    c->ops->momentum_field(c);  // rho u at time t
    cudaMemsetAsync(B.lJF, 0, 3 * c->N * sizeof(R), c->stream);
    const R* P = (const R*)c->P[c->pc];
    const R* H = (const R*)c->H[c->hc];
    const R* geo = (const R*)c->G[c->gc];
    const Mom4<R>* jf = (const Mom4<R>*)c->jf;
    k_adj_local<R><<<nb(c->N, TB_A), TB_A, 0, c->stream>>>(L, P, H, geo, jf, B.lP[lp], B.lH[lp], B, B.lH[dst]);
    k_adj_gather<R><<<nb(c->N, 256), 256, 0, c->stream>>>(L, H, geo, jf, B, B.lH[dst]);
    finish_step<R>(c, L, B, dst);
    c->adj.lp = dst;
}

template <class R> void init_back(cslbm_ctx* c)
{
    Lat L = make_lat(c);
    Bufs<R> B = bufs<R>(c);
    const int lp = c->adj.lp;
    k_adj_init<R><<<nb(c->N, 256), 256, 0, c->stream>>>(L, (const R*)c->G[c->gc], B.lP[lp], B.lH[lp], B.lGeo);
}

template <class R> void metric_grad(cslbm_ctx* c, const double* g6, const double* dg18, double* lg6, double* ldg18)
{
    Bufs<R> B = bufs<R>(c);
    k_adj_metric<R><<<nb(c->N, 128), 128, 0, c->stream>>>(c->N, g6, dg18, B.lGeo, lg6, ldg18);
}

}  // namespace adj
}  // namespace cslbm

namespace {

cslbm_status afail(cslbm_status s, const std::string& m) { return cslbm_record_error(s, m.c_str()); }

cslbm_status adj_ready(const cslbm_ctx* c)
{
    if (!c) return afail(CSLBM_EINVAL, "ctx is null");
    if (!c->adj.ws) return afail(CSLBM_ESTATE, "no adjoint workspace attached (cslbm_adjoint_attach)");
    if (!c->has_state) return afail(CSLBM_ESTATE, "no state");
    return CSLBM_OK;
}
cslbm_status launched(const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return afail(CSLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return CSLBM_OK;
}

}  // namespace

extern "C" {

cslbm_status cslbm_adjoint_workspace_bytes(const cslbm_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return afail(CSLBM_EINVAL, "null argument");
    if (c->p.storage != CSLBM_FP32 && c->p.storage != CSLBM_FP64)
        return afail(CSLBM_EINVAL, "the adjoint supports FP32 and FP64 storage");
    for (int a = 0; a < 3; a++)
        if ((c->p.bc_lo[a] != CSLBM_PERIODIC && c->p.bc_lo[a] != CSLBM_WALL) ||
            (c->p.bc_hi[a] != CSLBM_PERIODIC && c->p.bc_hi[a] != CSLBM_WALL))
            return afail(CSLBM_EINVAL, "the adjoint supports periodic faces and walls only");
    *bytes = cslbm::adj::adj_bytes(c);
    return CSLBM_OK;
}

cslbm_status cslbm_adjoint_attach(cslbm_ctx* c, void* workspace, size_t bytes)
{
    size_t need = 0;
    if (cslbm_status s = cslbm_adjoint_workspace_bytes(c, &need)) return s;
    if (!workspace || bytes < need) return afail(CSLBM_ENOMEM, "adjoint workspace smaller than required");
    if ((uintptr_t)workspace & 255) return afail(CSLBM_EINVAL, "adjoint workspace must be 256-byte aligned");
    c->adj.ws = workspace;
    c->adj.lp = 0;
    if (cudaMemsetAsync(workspace, 0, need, c->stream) != cudaSuccess) return afail(CSLBM_ECUDA, "memset failed");
    return CSLBM_OK;
}

cslbm_status cslbm_adjoint_seed_wall_force(cslbm_ctx* c, int axis, int side, const double e3[3])
{
    if (cslbm_status s = adj_ready(c)) return s;
    if (axis < 0 || axis > 2 || side < 0 || side > 1 || !e3) return afail(CSLBM_EINVAL, "bad argument");
    if ((side ? c->p.bc_hi[axis] : c->p.bc_lo[axis]) != CSLBM_WALL) return afail(CSLBM_EINVAL, "face is not a wall");
    if (c->p.storage == CSLBM_FP64) cslbm::adj::seed<double>(c, axis, side, e3);
    else cslbm::adj::seed<float>(c, axis, side, e3);
    return launched("adjoint seed");
}

cslbm_status cslbm_step_backward(cslbm_ctx* c)
{
    if (cslbm_status s = adj_ready(c)) return s;
    if (c->p.storage == CSLBM_FP64) cslbm::adj::backward<double>(c);
    else cslbm::adj::backward<float>(c);
    c->launches += 6;
    return launched("adjoint step");
}

cslbm_status cslbm_adjoint_init_backward(cslbm_ctx* c)
{
    if (cslbm_status s = adj_ready(c)) return s;
    if (c->p.storage == CSLBM_FP64) cslbm::adj::init_back<double>(c);
    else cslbm::adj::init_back<float>(c);
    return launched("adjoint initialisation");
}

cslbm_status cslbm_adjoint_metric_grad(cslbm_ctx* c, const double* g6, const double* dg18, double* grad_g6,
                                       double* grad_dg18, double* grad_J9)
{
    if (cslbm_status s = adj_ready(c)) return s;
    if (!g6 || !dg18 || !grad_g6 || !grad_dg18) return afail(CSLBM_EINVAL, "null argument");
    if (c->p.storage == CSLBM_FP64) cslbm::adj::metric_grad<double>(c, g6, dg18, grad_g6, grad_dg18);
    else cslbm::adj::metric_grad<float>(c, g6, dg18, grad_g6, grad_dg18);
    if (grad_J9) {
        const char* p = (const char*)c->adj.ws + cslbm::adj::adj_bytes(c) - ((9 * (size_t)c->N * 8 + 63) / 64 * 64);
        if (cudaMemcpyAsync(grad_J9, p, 9 * (size_t)c->N * 8, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            return afail(CSLBM_ECUDA, "copy failed");
    }
    return launched("adjoint metric");
}

}  // extern "C"
