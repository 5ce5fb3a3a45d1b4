// LBM step as two flat passes per time step.
//
// The forcing moment C^ij (Eq. forcing-C) needs the lattice gradient of
// rho u at time t on the 18 neighbours of every node (App. D).  The first
// pass forms rho u of every node (one float4 per node, a field small enough
// to stay in L2); the second pass steps every node independently: pull
// gather, moments, stress, gradient from the neighbours' rho u, forcing
// moments, collision, store.  No barriers and no shared memory, so the SMs
// run at the occupancy the registers allow; the price over the one-pass
// ideal is one extra read of the populations per step.
//
// Nodes on a non-periodic face take one generic out-of-line path (boundary
// rule, ghost extrapolation of the stencil); every other node has all its
// pull sources and stencil sites inside the domain after periodic wrapping.
#pragma once

#include "step_math.cuh"

namespace cslbm {

template <class R> struct alignas(4 * sizeof(R)) Mom4 {
    R x, y, z, w;
};

// 32-bit element offsets of a node's pull sources / stencil sites for
// c in {-1, 0, +1} per axis (the host guarantees 25 N < 2^32)
struct Nbr {
    unsigned xs[3], ys[3], zs[3];
};
__device__ __forceinline__ Nbr nbr_index(const Lat& L, int x, int y, int z, int sign)
{
    Nbr p;
    const unsigned n0 = L.n[0], n01 = (unsigned)L.n[0] * L.n[1];
#pragma unroll
    for (int c = -1; c <= 1; c++) {
        p.xs[c + 1] = (unsigned)wrapc(x + sign * c, L.n[0]);
        p.ys[c + 1] = (unsigned)wrapc(y + sign * c, L.n[1]) * n0;
        p.zs[c + 1] = (unsigned)wrapc(z + sign * c, L.n[2]) * n01;
    }
    return p;
}
__device__ __forceinline__ unsigned nbr_off(const Nbr& p, int cx, int cy, int cz)
{
    return p.zs[cz + 1] + p.ys[cy + 1] + p.xs[cx + 1];
}

// rho u of a boundary node from the boundary rule
template <class S, class R>
__device__ __noinline__ void momentum_boundary(const Lat& L, const S* __restrict__ P, const R* __restrict__ hist,
                                               const R* __restrict__ geo, int x, int y, int z, Mom4<R>* jf)
{
    R s[Q];
    boundary_pops<S, R>(L, P, hist, geo, x, y, z, s);
    PairSums<R> Ps;
    pair_sums(s, Ps);
    R m1[3];
    first_moment(Ps, m1);
    const long long v = nidx(L, x, y, z);
    const R sg = geo[v];
    Mom4<R> j;
    j.x = fmad(sg, m1[0], R(0.5) * hist[1 * L.N + v]);
    j.y = fmad(sg, m1[1], R(0.5) * hist[2 * L.N + v]);
    j.z = fmad(sg, m1[2], R(0.5) * hist[3 * L.N + v]);
    j.w = R(0);
    jf[v] = j;
}

// launch shape of both passes: blocks of 256 consecutive nodes of a plane
// (blockIdx.x), one grid row per plane (blockIdx.y)
constexpr int TB = 256;

__device__ __forceinline__ bool flat_node(const Lat& L, int& x, int& y, int& z, unsigned& v)
{
    const unsigned n01 = (unsigned)L.n[0] * L.n[1];
    const unsigned r = blockIdx.x * (unsigned)TB + threadIdx.x;
    if (r >= n01) return false;
    y = (int)(r / (unsigned)L.n[0]);
    x = (int)(r - (unsigned)y * L.n[0]);
    z = blockIdx.y;
    v = (unsigned)z * n01 + r;
    return true;
}

// rho u of one node into jf[v] (pull gather; boundary rule on face nodes)
template <class S, class R>
__device__ __forceinline__ void momentum_node(const Lat& L, const S* __restrict__ P, const R* __restrict__ hist,
                                              const R* __restrict__ geo, Mom4<R>* __restrict__ jf, int x, int y,
                                              int z, unsigned v)
{
    const unsigned N = (unsigned)L.N;
    if (on_boundary(L, x, y, z)) {
        momentum_boundary<S, R>(L, P, hist, geo, x, y, z, jf);
        return;
    }
    const Nbr src = nbr_index(L, x, y, z, -1);
    R s[Q];
#pragma unroll
    for (int l = 0; l < Q; l++)
        s[l] = R(Store<S>::ld(P + (unsigned)pslot(l) * N + nbr_off(src, cvec(l, 0), cvec(l, 1), cvec(l, 2))));
    PairSums<R> Ps;
    pair_sums(s, Ps);
    R m1[3];
    first_moment(Ps, m1);
    const R sg = __ldg(geo + v);
    Mom4<R> j;
    j.x = fmad(sg, m1[0], R(0.5) * __ldg(hist + 1 * N + v));
    j.y = fmad(sg, m1[1], R(0.5) * __ldg(hist + 2 * N + v));
    j.z = fmad(sg, m1[2], R(0.5) * __ldg(hist + 3 * N + v));
    j.w = R(0);
    jf[v] = j;
}

template <class S, class R>
__global__ void __launch_bounds__(TB) k_momentum_flat(Lat L, const S* __restrict__ P, const R* __restrict__ hist,
                                                      const R* __restrict__ geo, Mom4<R>* __restrict__ jf)
{
    int x, y, z;
    unsigned v;
    if (!flat_node(L, x, y, z, v)) return;
    momentum_node<S, R>(L, P, hist, geo, jf, x, y, z, v);
}

// rho u at a stencil site that may lie one step outside a non-periodic face:
// linear extrapolation 2 j(face) - j(face - normal) per out-of-range axis
// (tensor product over the axes).  Each axis contributes one or two
// (coordinate, weight) terms; the 2 x 2 x 2 sum is unrolled with the loads of
// zero-weight terms predicated off, so that all loads can be in flight at once.
__device__ __forceinline__ void site_axis(int r, int n, bool per_lo, bool per_hi, int& c0, int& c1, float& w0, float& w1)
{
    if (r >= 0 && r < n) { c0 = c1 = r; w0 = 1.0f; w1 = 0.0f; }
    else if (r < 0 && per_lo) { c0 = c1 = r + n; w0 = 1.0f; w1 = 0.0f; }
    else if (r >= n && per_hi) { c0 = c1 = r - n; w0 = 1.0f; w1 = 0.0f; }
    else if (r < 0) { c0 = 0; c1 = 1; w0 = 2.0f; w1 = -1.0f; }
    else { c0 = n - 1; c1 = n - 2; w0 = 2.0f; w1 = -1.0f; }
}
template <class R>
__device__ __forceinline__ Mom4<R> mom_site(const Lat& L, const Mom4<R>* __restrict__ jf, int x, int y, int z)
{
    // most sites of a face node's stencil are lattice nodes (after a periodic
    // wrap): one load, the value the weighted sum below would give
    {
        const int r[3] = {x, y, z};
        int w[3];
        bool ghost = false;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            w[a] = r[a];
            if (r[a] < 0) {
                if (L.bclo[a] == BC_PERIODIC) w[a] += L.n[a];
                else ghost = true;
            } else if (r[a] >= L.n[a]) {
                if (L.bchi[a] == BC_PERIODIC) w[a] -= L.n[a];
                else ghost = true;
            }
        }
        if (!ghost) return jf[((unsigned)w[2] * L.n[1] + w[1]) * (unsigned)L.n[0] + w[0]];
    }
    int x0, x1, y0, y1, z0, z1;
    float wx0, wx1, wy0, wy1, wz0, wz1;
    site_axis(x, L.n[0], L.bclo[0] == BC_PERIODIC, L.bchi[0] == BC_PERIODIC, x0, x1, wx0, wx1);
    site_axis(y, L.n[1], L.bclo[1] == BC_PERIODIC, L.bchi[1] == BC_PERIODIC, y0, y1, wy0, wy1);
    site_axis(z, L.n[2], L.bclo[2] == BC_PERIODIC, L.bchi[2] == BC_PERIODIC, z0, z1, wz0, wz1);
    Mom4<R> acc;
    acc.x = acc.y = acc.z = acc.w = R(0);
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = 0; k < 2; k++)
#pragma unroll
            for (int m = 0; m < 2; m++) {
                const float w = (i ? wx1 : wx0) * (k ? wy1 : wy0) * (m ? wz1 : wz0);
                if (w != 0.0f) {
                    const Mom4<R> j = jf[nidx(L, i ? x1 : x0, k ? y1 : y0, m ? z1 : z0)];
                    acc.x += R(w) * j.x;
                    acc.y += R(w) * j.y;
                    acc.z += R(w) * j.z;
                }
            }
    return acc;
}

// L2 eviction policies (createpolicy): data read or written once per step
// goes out of L2 first; data read again within the step stays longer
__device__ __forceinline__ unsigned long long policy_evict_first()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long policy_evict_last()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
// a store carrying an L2 eviction policy
__device__ __forceinline__ void st_hint(float* p, float v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;\n" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(double* p, double v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;\n" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(__half* p, float v, unsigned long long pol)
{
    const unsigned short b = __half_as_ushort(__float2half_rn(v));
    asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;\n" ::"l"(p), "h"(b), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(__nv_bfloat16* p, float v, unsigned long long pol)
{
    const unsigned short b = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;\n" ::"l"(p), "h"(b), "l"(pol) : "memory");
}

// the step of one node from its populations s (h - w), geometry and history
// at element offset v, and the rho u differences d across the nine opposite
// stencil pairs; stores the new populations and forcing coefficients (with
// the L2 policy pol when HINT)
template <class S, class R, bool HINT = false>
__device__ __forceinline__ void step_core(const Lat& L, const R s[Q], const GeoT<R>& G, const HistT<R>& Hp,
                                          const R d[9][3], S* __restrict__ Pout, R* __restrict__ hout, unsigned v,
                                          unsigned N, unsigned long long pol = 0)
{
    PairSums<R> Ps;
    pair_sums(s, Ps);
    R m0, m1[3], m2[6];
    all_moments(s, Ps, m0, m1, m2);
    const R rho = fmad(G.sg, m0 + R(1), R(0.5) * Hp.A);
    const R ir = recip(rho);
    R j[3];
#pragma unroll
    for (int a = 0; a < 3; a++) j[a] = fmad(G.sg, m1[a], R(0.5) * Hp.B[a]);
    R Tt[6];
    stress_t<R, R>(R(L.theta), R(L.kvisc), G, rho, ir, j, m2, Hp, Tt);
    R D[3][3];
    gradient_from_pairs(d, D);
    const R fext[3] = {R(L.fext[0]), R(L.fext[1]), R(L.fext[2])};
    HistT<R> H;
    forcing_t<R, R>(R(L.theta), fext, G, j, Tt, D, H);
    R out[Q];
    collide_t<R, R>(R(L.omega), R(L.theta), G, s, m0, rho, ir, j, Hp, H, out);
    if constexpr (HINT) {
        st_hint(hout + v, H.A, pol);
#pragma unroll
        for (int a = 0; a < 3; a++) st_hint(hout + (1 + a) * N + v, H.B[a], pol);
#pragma unroll
        for (int a = 0; a < 6; a++) st_hint(hout + (4 + a) * N + v, H.C[a], pol);
#pragma unroll
        for (int l = 0; l < Q; l++) st_hint(Pout + (unsigned)pslot(l) * N + v, out[l], pol);
    } else {
        hout[v] = H.A;
#pragma unroll
        for (int a = 0; a < 3; a++) hout[(1 + a) * N + v] = H.B[a];
#pragma unroll
        for (int a = 0; a < 6; a++) hout[(4 + a) * N + v] = H.C[a];
#pragma unroll
        for (int l = 0; l < Q; l++) Store<S>::st(Pout + (unsigned)pslot(l) * N + v, out[l]);
    }
}

template <class R>
__device__ __forceinline__ void load_geo_hist(const R* __restrict__ geo, const R* __restrict__ hist, unsigned v,
                                              unsigned N, GeoT<R>& G, HistT<R>& Hp)
{
    G.sg = __ldg(geo + v);
    G.isg = recip(G.sg);
#pragma unroll
    for (int a = 0; a < 6; a++) G.gi[a] = __ldg(geo + (1 + a) * N + v);
#pragma unroll
    for (int a = 0; a < 18; a++) G.gam[a] = __ldg(geo + (7 + a) * N + v);
#pragma unroll
    for (int k = 0; k < 3; k++) G.gc[k] = (G.gam[0 * 6 + s6(k, 0)] + G.gam[1 * 6 + s6(k, 1)]) + G.gam[2 * 6 + s6(k, 2)];
    Hp.A = __ldg(hist + v);
#pragma unroll
    for (int a = 0; a < 3; a++) Hp.B[a] = __ldg(hist + (1 + a) * N + v);
#pragma unroll
    for (int a = 0; a < 6; a++) Hp.C[a] = __ldg(hist + (4 + a) * N + v);
}

// the step of a node on a non-periodic face (boundary rule, ghost stencil)
template <class S, class R>
__device__ __forceinline__ void step_boundary_body(const Lat& L, const S* __restrict__ Pin, S* __restrict__ Pout,
                                                   const R* __restrict__ hin, R* __restrict__ hout,
                                                   const R* __restrict__ geo, const Mom4<R>* __restrict__ jf, int x,
                                                   int y, int z)
{
    const unsigned N = (unsigned)L.N, v = (unsigned)nidx(L, x, y, z);
    GeoT<R> G;
    HistT<R> Hp;
    load_geo_hist(geo, hin, v, N, G, Hp);
    // the boundary rule with the node's own metric and history as loaded
    Geo<R> Gw;
    Gw.sg = G.sg;
    Gw.isg = G.isg;
#pragma unroll
    for (int a = 0; a < 6; a++) Gw.gi[a] = G.gi[a];
    Hist<R> Hw;
    Hw.A = Hp.A;
#pragma unroll
    for (int a = 0; a < 3; a++) Hw.B[a] = Hp.B[a];
#pragma unroll
    for (int a = 0; a < 6; a++) Hw.C[a] = Hp.C[a];
    R s[Q];
    boundary_pops_w<S, R>(L, Pin, hin, geo, x, y, z, Gw, Hw, s);
    R d[9][3];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const int l = 2 * k + 1, cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
        const Mom4<R> p = mom_site(L, jf, x + cx, y + cy, z + cz), m = mom_site(L, jf, x - cx, y - cy, z - cz);
        d[k][0] = p.x - m.x;
        d[k][1] = p.y - m.y;
        d[k][2] = p.z - m.z;
    }
    step_core<S, R>(L, s, G, Hp, d, Pout, hout, v, N);
}

// out of line where face nodes share a kernel with interior nodes
template <class S, class R>
__device__ __noinline__ void step_boundary(const Lat& L, const S* __restrict__ Pin, S* __restrict__ Pout,
                                           const R* __restrict__ hin, R* __restrict__ hout, const R* __restrict__ geo,
                                           const Mom4<R>* __restrict__ jf, int x, int y, int z)
{
    step_boundary_body<S, R>(L, Pin, Pout, hin, hout, geo, jf, x, y, z);
}

// the step of one node: pull gather, moments, gradient from the rho u field,
// forcing, collision, store (the boundary rule and ghost stencil out of line
// on face nodes)
template <class S, class R>
__device__ __forceinline__ void step_node(const Lat& L, const S* __restrict__ Pin, S* __restrict__ Pout,
                                          const R* __restrict__ hin, R* __restrict__ hout, const R* __restrict__ geo,
                                          const Mom4<R>* __restrict__ jf, int x, int y, int z, unsigned v)
{
    const unsigned N = (unsigned)L.N;
    if (on_boundary(L, x, y, z)) {
        step_boundary<S, R>(L, Pin, Pout, hin, hout, geo, jf, x, y, z);
        return;
    }
    const Nbr src = nbr_index(L, x, y, z, -1);
    R s[Q];
#pragma unroll
    for (int l = 0; l < Q; l++)
        s[l] = R(Store<S>::ld(Pin + (unsigned)pslot(l) * N + nbr_off(src, cvec(l, 0), cvec(l, 1), cvec(l, 2))));
    GeoT<R> G;
    HistT<R> Hp;
    load_geo_hist(geo, hin, v, N, G, Hp);
    const Nbr nb = nbr_index(L, x, y, z, +1);  // sites x + c
    R d[9][3];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const int l = 2 * k + 1, cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
        const Mom4<R> p = jf[nbr_off(nb, cx, cy, cz)], m = jf[nbr_off(nb, -cx, -cy, -cz)];
        d[k][0] = p.x - m.x;
        d[k][1] = p.y - m.y;
        d[k][2] = p.z - m.z;
    }
    step_core<S, R>(L, s, G, Hp, d, Pout, hout, v, N);
}

template <class S, class R>
__global__ void __launch_bounds__(TB, 2) k_step_flat(Lat L, const S* __restrict__ Pin, S* __restrict__ Pout,
                                                     const R* __restrict__ hin, R* __restrict__ hout,
                                                     const R* __restrict__ geo, const Mom4<R>* __restrict__ jf)
{
    int x, y, z;
    unsigned v;
    if (!flat_node(L, x, y, z, v)) return;
    step_node<S, R>(L, Pin, Pout, hin, hout, geo, jf, x, y, z, v);
}

// The nodes on non-periodic faces as up to six boxes without overlap: the
// faces of axis 2 whole, those of axis 1 without the axis-2 face nodes, those
// of axis 0 without the face nodes of axes 1 and 2.
struct FaceList {
    int nseg;
    int lo[6][3], len[6][3];
    long long start[7];
};

inline FaceList face_list(const cslbm_ctx* c)
{
    FaceList f{};
    long long total = 0;
    bool done[3] = {false, false, false};
    for (int a = 2; a >= 0; a--) {
        if (c->p.bc_lo[a] == CSLBM_PERIODIC) continue;
        for (int side = 0; side < 2; side++) {
            const int k = f.nseg++;
            for (int b = 0; b < 3; b++) {
                if (b == a) {
                    f.lo[k][b] = side ? c->n[b] - 1 : 0;
                    f.len[k][b] = 1;
                } else if (done[b]) {
                    f.lo[k][b] = 1;
                    f.len[k][b] = c->n[b] - 2;
                } else {
                    f.lo[k][b] = 0;
                    f.len[k][b] = c->n[b];
                }
            }
            f.start[k] = total;
            total += (long long)f.len[k][0] * f.len[k][1] * f.len[k][2];
        }
        done[a] = true;
    }
    f.start[f.nseg] = total;
    return f;
}

// one step of the face nodes only (the interior comes from the row-staged pass)
template <class S, class R>
__global__ void __launch_bounds__(128) k_step_faces(const __grid_constant__ Lat L, const __grid_constant__ FaceList f,
                                                    const S* __restrict__ Pin, S* __restrict__ Pout,
                                                    const R* __restrict__ hin, R* __restrict__ hout,
                                                    const R* __restrict__ geo, const Mom4<R>* __restrict__ jf)
{
    // face nodes number fewer than 2^31 (the lattice's nodes do)
    const int i = blockIdx.x * 128 + threadIdx.x;
    if (i >= (int)f.start[f.nseg]) return;
    // segment of node i, by selects over the six (no indexing of f by a
    // runtime value, which would copy it to local memory)
    int lo0 = 0, lo1 = 0, lo2 = 0, len0 = 1, len1 = 1, st = 0;
#pragma unroll
    for (int k = 0; k < 6; k++)
        if (k < f.nseg && i >= (int)f.start[k]) {
            lo0 = f.lo[k][0];
            lo1 = f.lo[k][1];
            lo2 = f.lo[k][2];
            len0 = f.len[k][0];
            len1 = f.len[k][1];
            st = (int)f.start[k];
        }
    const int r = i - st, q = r / len0;
    const int x = lo0 + (r - q * len0);
    const int y = lo1 + q % len1;
    const int z = lo2 + q / len1;
    step_boundary_body<S, R>(L, Pin, Pout, hin, hout, geo, jf, x, y, z);
}

template <class S, class R>
int launch_faces(const cslbm_ctx* c, const Lat& L, const S* Pin, S* Pout, const R* hin, R* hout, const R* geo,
                 cudaStream_t stream)
{
    const FaceList f = face_list(c);
    const long long total = f.start[f.nseg];
    if (total == 0) return 0;
    k_step_faces<S, R><<<(unsigned)((total + 127) / 128), 128, 0, stream>>>(L, f, Pin, Pout, hin, hout, geo,
                                                                               (const Mom4<R>*)c->jf);
    return 1;
}

inline dim3 flat_grid(const cslbm_ctx* c)
{
    return dim3((unsigned)(((long long)c->n[0] * c->n[1] + TB - 1) / TB), c->n[2]);
}

template <class S, class R>
void launch_momentum(const cslbm_ctx* c, const Lat& L, const S* P, const R* hin, const R* geo)
{
    k_momentum_flat<S, R><<<flat_grid(c), TB, 0, c->stream>>>(L, P, hin, geo, (Mom4<R>*)c->jf);
}

// one time step: momentum pass, then the step pass
template <class S, class R>
void launch_flat_step(const cslbm_ctx* c, const Lat& L, const S* Pin, S* Pout, const R* hin, R* hout, const R* geo)
{
    launch_momentum<S, R>(c, L, Pin, hin, geo);
    k_step_flat<S, R><<<flat_grid(c), TB, 0, c->stream>>>(L, Pin, Pout, hin, hout, geo,
                                                                         (const Mom4<R>*)c->jf);
}

}  // namespace cslbm
