// Fused LBM step: one kernel per time step.
//
// The forcing moment C^ij (Eq. forcing-C) needs the lattice gradient of
// rho u at time t on the 18 neighbours of every node (App. D), i.e. the
// momentum of the whole neighbourhood before any node can collide.  Instead
// of writing a momentum field to HBM and reading it back, each CTA owns a
// 32 x 8 column of the lattice and marches along axis 2.  For every plane it
// gathers the populations of its nodes plus a one-node ring around the tile,
// forms rho u there into a four-plane ring buffer in shared memory, and then
// steps the plane below.  The ring costs extra L2 reads (its populations
// belong to neighbouring tiles), not extra DRAM traffic: per node update the
// kernel moves the algorithmic 19 + 19 populations, 10 + 10 history
// coefficients and 25 geometry values.
//
// Each thread steps two x-adjacent nodes with packed FP32 arithmetic
// (step_math.cuh); the geometry and history of the plane being stepped are
// copied to shared memory with cp.async while the next plane is gathered.
// Each thread only reads back its own copies and its own gathered
// populations, so the two barriers per plane guard only the momentum buffer.
//
// Stencil sites outside a non-periodic face take the linear extrapolation
// 2 j(face) - j(face - normal) per out-of-range axis.  Boundary nodes take
// the boundary rule out of line (they are whole planes or whole rows when
// the non-periodic faces sit on axes 1 and 2).
#pragma once

#include "step_math.cuh"

namespace cslbm {

constexpr int FX = 32, FY = 8, FP = FX / 2;  // tile, node pairs per row
constexpr int FT = FP * FY;                   // threads per CTA (one per pair)
constexpr int EX = FX + 2, EY = FY + 2;       // tile with its ring
constexpr int NPRE = NGEO + NHIST;            // prefetched values per node
constexpr int JSLOTS = 4;

// rho u of one site (x, y, z, unused), one vector load per site
template <class R> struct alignas(4 * sizeof(R)) J4 {
    R x, y, z, w;
};
template <class R> struct Vec4 {
    using type = J4<R>;
};

template <class R> struct FusedSmem {
    R s[2][Q][FY][FX];                         // populations (h - w) of planes z, z+1
    typename Vec4<R>::type j[JSLOTS][EY][EX];  // rho u (x, y, z, unused) of four planes
    R pre[NPRE][FY][FX];                       // geometry and history of plane z
};

__device__ __forceinline__ int jslot(int z) { return z & (JSLOTS - 1); }  // two's complement: -1 -> 3

// asynchronous global -> shared copy of 4, 8 or 16 bytes
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// paired loads and stores of two consecutive elements (vector access when
// the pair is aligned)
template <class S, class R> struct PairIO;
template <> struct PairIO<float, float> {
    static __device__ __forceinline__ Pair<float> ld(const float* p, bool vec)
    {
        return vec ? Pair<float>(__ldg(reinterpret_cast<const float2*>(p))) : Pair<float>(__ldg(p), __ldg(p + 1));
    }
    static __device__ __forceinline__ void st(float* p, Pair<float> v, bool vec, bool both)
    {
        if (vec && both) *reinterpret_cast<float2*>(p) = v.v;
        else {
            p[0] = v.lo();
            if (both) p[1] = v.hi();
        }
    }
};
template <> struct PairIO<double, double> {
    static __device__ __forceinline__ Pair<double> ld(const double* p, bool vec)
    {
        if (vec) {
            const double2 t = __ldg(reinterpret_cast<const double2*>(p));
            return Pair<double>(t.x, t.y);
        }
        return Pair<double>(__ldg(p), __ldg(p + 1));
    }
    static __device__ __forceinline__ void st(double* p, Pair<double> v, bool vec, bool both)
    {
        if (vec && both) *reinterpret_cast<double2*>(p) = make_double2(v.x, v.y);
        else {
            p[0] = v.x;
            if (both) p[1] = v.y;
        }
    }
};
template <> struct PairIO<__half, float> {
    static __device__ __forceinline__ Pair<float> ld(const __half* p, bool vec)
    {
        if (vec) return Pair<float>(__half22float2(__ldg(reinterpret_cast<const __half2*>(p))));
        return Pair<float>(__half2float(__ldg(p)), __half2float(__ldg(p + 1)));
    }
    static __device__ __forceinline__ void st(__half* p, Pair<float> v, bool vec, bool both)
    {
        if (vec && both) *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.lo(), v.hi());
        else {
            p[0] = __float2half_rn(v.lo());
            if (both) p[1] = __float2half_rn(v.hi());
        }
    }
};
template <> struct PairIO<__nv_bfloat16, float> {
    static __device__ __forceinline__ Pair<float> ld(const __nv_bfloat16* p, bool vec)
    {
        if (vec) return Pair<float>(__bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p))));
        return Pair<float>(__bfloat162float(__ldg(p)), __bfloat162float(__ldg(p + 1)));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, Pair<float> v, bool vec, bool both)
    {
        if (vec && both) *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.lo(), v.hi());
        else {
            p[0] = __float2bfloat16_rn(v.lo());
            if (both) p[1] = __float2bfloat16_rn(v.hi());
        }
    }
};

// a pair into two consecutive shared-memory entries (8- or 16-byte aligned)
__device__ __forceinline__ void st_pair_smem(float* p, Pair<float> v) { *reinterpret_cast<float2*>(p) = v.v; }
__device__ __forceinline__ void st_pair_smem(double* p, Pair<double> v) { *reinterpret_cast<double2*>(p) = make_double2(v.x, v.y); }
__device__ __forceinline__ Pair<float> ld_pair_smem(const float* p) { return Pair<float>(*reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ Pair<double> ld_pair_smem(const double* p)
{
    const double2 t = *reinterpret_cast<const double2*>(p);
    return Pair<double>(t.x, t.y);
}

// m1 = sum s c for one node (scalar)
template <class R>
__device__ __forceinline__ void sum_m1(const R s[Q], R m1[3])
{
    PairSums<R> P;
    pair_sums(s, P);
    first_moment(P, m1);
}

template <class R, class V4> __device__ __forceinline__ void put_j(V4* dst, R jx, R jy, R jz)
{
    V4 v;
    v.x = jx;
    v.y = jy;
    v.z = jz;
    v.w = R(0);
    *dst = v;
}

// One site of the tile or ring taken node by node: populations through the
// boundary rule when the node is on a non-periodic face, else the raw pull
// gather; rho u into jdst and, when sdst is given, the populations into the
// plane buffer (stride ss).  Out of line: the common path stays in registers.
template <class S, class R, class V4>
__device__ __noinline__ void scalar_site(const Lat& L, const S* __restrict__ P, const R* __restrict__ hist,
                                         const R* __restrict__ geo, int x, int y, int z, V4* jdst, R* sdst, int ss)
{
    R s[Q], m1[3];
    node_pops<S, R>(L, P, hist, geo, x, y, z, s);
    sum_m1(s, m1);
    const long long v = nidx(L, x, y, z);
    const R sg = geo[v];
    put_j<R>(jdst, sg * m1[0] + R(0.5) * hist[1 * L.N + v], sg * m1[1] + R(0.5) * hist[2 * L.N + v],
             sg * m1[2] + R(0.5) * hist[3 * L.N + v]);
    if (sdst)
        for (int l = 0; l < Q; l++) sdst[l * ss] = s[l];
}

template <class S, class R>
__global__ void __launch_bounds__(FT, sizeof(R) == 4 ? 2 : 1)
    k_step_fused(Lat L, const S* __restrict__ Pin, S* __restrict__ Pout, const R* __restrict__ hin,
                 R* __restrict__ hout, const R* __restrict__ geo, int zc)
{
    using V4 = typename Vec4<R>::type;
    using T = Pair<R>;
    using IO = PairIO<S, R>;
    using GIO = PairIO<R, R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem<R>& sm = *reinterpret_cast<FusedSmem<R>*>(smem_raw);
    const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
    const unsigned N = (unsigned)L.N, n01 = (unsigned)n0 * n1;
    const int tid = threadIdx.x, px = tid % FP, ty = tid / FP, tx = 2 * px;
    const int ntx = (n0 + FX - 1) / FX;
    const int x0 = (blockIdx.x % ntx) * FX, y0 = (blockIdx.x / ntx) * FY;
    const int w = min(FX, n0 - x0), h = min(FY, n1 - y0);
    const int z0 = blockIdx.y * zc, z1 = min(n2, z0 + zc);
    const bool act = tx < w && ty < h;       // first node of the pair
    const bool both = act && tx + 1 < w;     // second node too
    const int x = x0 + tx, y = y0 + ty;
    const bool vec = (n0 & 1) == 0;          // pairs start on even elements
    const bool xper = L.bclo[0] == BC_PERIODIC, yper = L.bclo[1] == BC_PERIODIC, zper = L.bclo[2] == BC_PERIODIC;

    // ring site of this thread: bottom row, top row, left column, right column
    const int nring = 2 * (w + 2) + 2 * h;
    int rx, ry;
    if (tid < w + 2) { rx = tid; ry = 0; }
    else if (tid < 2 * (w + 2)) { rx = tid - (w + 2); ry = h + 1; }
    else if (tid < 2 * (w + 2) + h) { rx = 0; ry = tid - 2 * (w + 2) + 1; }
    else { rx = w + 1; ry = tid - 2 * (w + 2) - h + 1; }
    const bool has_ring = tid < nring;
    int gx = x0 - 1 + rx, gy = y0 - 1 + ry;
    const bool xout = gx < 0 || gx >= n0, yout = gy < 0 || gy >= n1;
    const bool rghost = (xout && !xper) || (yout && !yper);
    if (xout && xper) gx = wrapc(gx, n0);
    if (yout && yper) gy = wrapc(gy, n1);

    auto inplane = [&](int zz, int& zw) {
        zw = zz;
        if (zz >= 0 && zz < n2) return true;
        if (!zper) return false;
        zw = wrapc(zz, n2);
        return true;
    };

    // populations of plane zz into s[buf] and rho u into the momentum buffer
    auto gather_plane = [&](int zz, int buf) {
        int zw;
        if (!inplane(zz, zw)) return;
        const int sl = jslot(zz);
        if (act) {
            const int xb = both ? x + 1 : x;
            if (!on_boundary(L, x, y, zw) && !on_boundary(L, xb, y, zw)) {
                // x coordinates of the sources: x+1, x, x-1 for the first node,
                // x+2, x+1, x for the second (source = node - c)
                const unsigned xa[3] = {(unsigned)wrapc(x + 1, n0), (unsigned)x, (unsigned)wrapc(x - 1, n0)};
                const unsigned xc[3] = {(unsigned)wrapc(xb + 1, n0), (unsigned)xb, (unsigned)wrapc(xb - 1, n0)};
                unsigned ys[3], zs[3];
#pragma unroll
                for (int c = -1; c <= 1; c++) {
                    ys[c + 1] = (unsigned)wrapc(y - c, n1) * (unsigned)n0;
                    zs[c + 1] = (unsigned)wrapc(zw - c, n2) * n01;
                }
                T s[Q];
#pragma unroll
                for (int l = 0; l < Q; l++) {
                    const int cx = cvec(l, 0);
                    const unsigned base = (unsigned)l * N + zs[cvec(l, 2) + 1] + ys[cvec(l, 1) + 1];
                    if (cx == 0 && both) s[l] = IO::ld(Pin + base + x, vec);
                    else s[l] = T(R(Store<S>::ld(Pin + base + xa[cx + 1])), R(Store<S>::ld(Pin + base + xc[cx + 1])));
                }
                PairSums<T> Ps;
                pair_sums(s, Ps);
                T m1[3];
                first_moment(Ps, m1);
                const unsigned v = n01 * zw + (unsigned)n0 * y + x, vb = both ? v + 1 : v;
                auto ld2 = [&](const R* p) { return both ? GIO::ld(p + v, vec) : T(__ldg(p + v)); };
                const T sg = ld2(geo);
                T jj[3];
#pragma unroll
                for (int a = 0; a < 3; a++) jj[a] = fmad(sg, m1[a], T(R(0.5)) * ld2(hin + (1 + a) * N));
                (void)vb;
                put_j<R>(&sm.j[sl][ty + 1][tx + 1], jj[0].lo(), jj[1].lo(), jj[2].lo());
                if (both) put_j<R>(&sm.j[sl][ty + 1][tx + 2], jj[0].hi(), jj[1].hi(), jj[2].hi());
#pragma unroll
                for (int l = 0; l < Q; l++) st_pair_smem(&sm.s[buf][l][ty][tx], s[l]);
            } else {
                scalar_site<S, R, V4>(L, Pin, hin, geo, x, y, zw, &sm.j[sl][ty + 1][tx + 1], &sm.s[buf][0][ty][tx],
                                      FY * FX);
                if (both)
                    scalar_site<S, R, V4>(L, Pin, hin, geo, xb, y, zw, &sm.j[sl][ty + 1][tx + 2],
                                          &sm.s[buf][0][ty][tx + 1], FY * FX);
            }
        }
        if (has_ring && !rghost) {
            if (on_boundary(L, gx, gy, zw)) {
                scalar_site<S, R, V4>(L, Pin, hin, geo, gx, gy, zw, &sm.j[sl][ry][rx], (R*)nullptr, 0);
            } else {
                R s[Q], m1[3];
                gather_raw<S, R>(L, Pin, gx, gy, zw, s);
                sum_m1(s, m1);
                const unsigned v = n01 * zw + (unsigned)n0 * gy + gx;
                const R sg = __ldg(geo + v);
                put_j<R>(&sm.j[sl][ry][rx], fmad(sg, m1[0], R(0.5) * __ldg(hin + 1 * N + v)),
                         fmad(sg, m1[1], R(0.5) * __ldg(hin + 2 * N + v)), fmad(sg, m1[2], R(0.5) * __ldg(hin + 3 * N + v)));
            }
        }
    };

    // ring sites outside a non-periodic x or y face of an in-domain plane
    auto fill_xy_ghosts = [&](int zz) {
        int zw;
        if (!inplane(zz, zw)) return;
        if (!(has_ring && rghost)) return;
        const int sl = jslot(zz);
        int cx0 = rx, cx1 = rx, cy0 = ry, cy1 = ry, nx = 1, ny = 1;
        if (xout && !xper) {
            nx = 2;
            if (gx < 0) { cx0 = 1; cx1 = 2; }
            else { cx0 = w; cx1 = w - 1; }
        }
        if (yout && !yper) {
            ny = 2;
            if (gy < 0) { cy0 = 1; cy1 = 2; }
            else { cy0 = h; cy1 = h - 1; }
        }
        R acc[3] = {R(0), R(0), R(0)};
        for (int i = 0; i < nx; i++)
            for (int k = 0; k < ny; k++) {
                const R wt = (i ? R(-1) : (nx == 2 ? R(2) : R(1))) * (k ? R(-1) : (ny == 2 ? R(2) : R(1)));
                const V4 jv = sm.j[sl][k ? cy1 : cy0][i ? cx1 : cx0];
                acc[0] += wt * jv.x;
                acc[1] += wt * jv.y;
                acc[2] += wt * jv.z;
            }
        put_j<R>(&sm.j[sl][ry][rx], acc[0], acc[1], acc[2]);
    };

    // a whole plane one step outside a non-periodic z face
    auto fill_z_ghost = [&](int zz) {
        const int sb = jslot(zz < 0 ? 0 : n2 - 1), si = jslot(zz < 0 ? 1 : n2 - 2), sl = jslot(zz);
        for (int k = tid; k < EY * EX; k += FT) {
            const V4 a = sm.j[sb][k / EX][k % EX], b = sm.j[si][k / EX][k % EX];
            put_j<R>(&sm.j[sl][k / EX][k % EX], R(2) * a.x - b.x, R(2) * a.y - b.y, R(2) * a.z - b.z);
        }
    };

    // geometry and history of plane zz into sm.pre (own entries)
    auto prefetch = [&](int zz) {
        if (act) {
            const unsigned v = n01 * zz + (unsigned)n0 * y + x;
            if (vec && both) {
#pragma unroll
                for (int k = 0; k < NGEO; k++) cp_async<2 * sizeof(R)>(&sm.pre[k][ty][tx], geo + k * N + v);
#pragma unroll
                for (int k = 0; k < NHIST; k++) cp_async<2 * sizeof(R)>(&sm.pre[NGEO + k][ty][tx], hin + k * N + v);
            } else {
#pragma unroll
                for (int k = 0; k < NGEO; k++) {
                    cp_async<sizeof(R)>(&sm.pre[k][ty][tx], geo + k * N + v);
                    if (both) cp_async<sizeof(R)>(&sm.pre[k][ty][tx + 1], geo + k * N + v + 1);
                }
#pragma unroll
                for (int k = 0; k < NHIST; k++) {
                    cp_async<sizeof(R)>(&sm.pre[NGEO + k][ty][tx], hin + k * N + v);
                    if (both) cp_async<sizeof(R)>(&sm.pre[NGEO + k][ty][tx + 1], hin + k * N + v + 1);
                }
            }
        }
        cp_async_commit();
    };
    auto pre = [&](int k) { return ld_pair_smem(&sm.pre[k][ty][tx]); };

    gather_plane(z0 - 1, 1);
    gather_plane(z0, 0);
    __syncthreads();
    fill_xy_ghosts(z0 - 1);
    fill_xy_ghosts(z0);

    for (int z = z0; z < z1; z++) {
        const int cur = (z - z0) & 1;
        prefetch(z);
        gather_plane(z + 1, cur ^ 1);
        __syncthreads();
        fill_xy_ghosts(z + 1);
        __syncthreads();
        if (!zper && (z == 0 || z == n2 - 1)) {
            if (z == 0) fill_z_ghost(-1);
            if (z == n2 - 1) fill_z_ghost(n2);
            __syncthreads();
        }
        cp_async_wait_all();
        if (act) {
            GeoT<T> G;
            G.sg = pre(0);
            G.isg = recip(G.sg);
#pragma unroll
            for (int a = 0; a < 6; a++) G.gi[a] = pre(1 + a);
#pragma unroll
            for (int a = 0; a < 18; a++) G.gam[a] = pre(7 + a);
#pragma unroll
            for (int k = 0; k < 3; k++) G.gc[k] = (G.gam[0 * 6 + s6(k, 0)] + G.gam[1 * 6 + s6(k, 1)]) + G.gam[2 * 6 + s6(k, 2)];
            HistT<T> Hp;
            Hp.A = pre(NGEO);
#pragma unroll
            for (int a = 0; a < 3; a++) Hp.B[a] = pre(NGEO + 1 + a);
#pragma unroll
            for (int a = 0; a < 6; a++) Hp.C[a] = pre(NGEO + 4 + a);
            T s[Q];
#pragma unroll
            for (int l = 0; l < Q; l++) s[l] = ld_pair_smem(&sm.s[cur][l][ty][tx]);
            PairSums<T> Ps;
            pair_sums(s, Ps);
            T m0, m1[3], m2[6];
            all_moments(s, Ps, m0, m1, m2);
            const T half(R(0.5));
            const T rho = fmad(G.sg, m0 + T(R(1)), half * Hp.A);
            const T ir = recip(rho);
            T j[3];
#pragma unroll
            for (int a = 0; a < 3; a++) j[a] = fmad(G.sg, m1[a], half * Hp.B[a]);
            T Tt[6];
            stress_t<T, R>(R(L.theta), R(L.kvisc), G, rho, ir, j, m2, Hp, Tt);
            // differences of rho u across the nine opposite directions
            T d[9][3];
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const int l = 2 * k + 1, cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
                const V4 pa = sm.j[jslot(z + cz)][ty + 1 + cy][tx + 1 + cx];
                const V4 pb = sm.j[jslot(z + cz)][ty + 1 + cy][tx + 2 + cx];
                const V4 ma = sm.j[jslot(z - cz)][ty + 1 - cy][tx + 1 - cx];
                const V4 mb = sm.j[jslot(z - cz)][ty + 1 - cy][tx + 2 - cx];
                d[k][0] = T(pa.x, pb.x) - T(ma.x, mb.x);
                d[k][1] = T(pa.y, pb.y) - T(ma.y, mb.y);
                d[k][2] = T(pa.z, pb.z) - T(ma.z, mb.z);
            }
            T D[3][3];
            gradient_from_pairs(d, D);
            R fext[3] = {R(L.fext[0]), R(L.fext[1]), R(L.fext[2])};
            HistT<T> H;
            forcing_t<T, R>(R(L.theta), fext, G, j, Tt, D, H);
            T out[Q];
            collide_t<T, R>(R(L.omega), R(L.theta), G, s, m0, rho, ir, j, Hp, H, out);
            const unsigned v = n01 * z + (unsigned)n0 * y + x;
            const bool vb = vec && both;
            GIO::st(hout + v, H.A, vb, both);
#pragma unroll
            for (int a = 0; a < 3; a++) GIO::st(hout + (1 + a) * N + v, H.B[a], vb, both);
#pragma unroll
            for (int a = 0; a < 6; a++) GIO::st(hout + (4 + a) * N + v, H.C[a], vb, both);
#pragma unroll
            for (int l = 0; l < Q; l++) IO::st(Pout + (unsigned)l * N + v, out[l], vb, both);
        }
    }
}

// grid: one CTA per (tile, chunk of planes); chunks sized so that about
// eight waves of two CTAs per SM are in flight
inline int fused_chunk(const cslbm_ctx* c)
{
    const int ntiles = ((c->n[0] + FX - 1) / FX) * ((c->n[1] + FY - 1) / FY);
    const int target = 8 * 2 * 152;
    int nch = (target + ntiles - 1) / ntiles;
    int zc = (c->n[2] + nch - 1) / nch;
    if (zc < 4) zc = 4;
    if (zc > c->n[2]) zc = c->n[2];
    return zc;
}

template <class S, class R>
void launch_fused_step(const cslbm_ctx* c, const Lat& L, const S* Pin, S* Pout, const R* hin, R* hout, const R* geo)
{
    const size_t smem = sizeof(FusedSmem<R>);
    cudaFuncSetAttribute(k_step_fused<S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int zc = fused_chunk(c);
    const unsigned ntiles = ((c->n[0] + FX - 1) / FX) * ((c->n[1] + FY - 1) / FY);
    dim3 grid(ntiles, (c->n[2] + zc - 1) / zc);
    k_step_fused<S, R><<<grid, FT, smem, c->stream>>>(L, Pin, Pout, hin, hout, geo, zc);
}

}  // namespace cslbm
