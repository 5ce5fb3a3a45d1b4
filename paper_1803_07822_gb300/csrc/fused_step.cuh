// Fused LBM step: one kernel per time step.
//
// The forcing moment C^ij (Eq. forcing-C) needs the lattice gradient of
// rho u at time t on the 18 neighbours of every node (App. D), i.e. the
// momentum of the whole neighbourhood before any node can collide.  Instead
// of writing a momentum field to HBM and reading it back, each CTA owns a
// 32 x 8 column of the lattice and marches along axis 2.  For every plane it
// gathers the populations of its nodes plus a one-node ring around the tile,
// forms rho u there into a three-plane ring buffer in shared memory, and then
// steps the plane below using the buffered populations.  The ring costs extra
// L2 reads (its populations belong to neighbouring tiles), not extra DRAM
// traffic: per node update the kernel moves the algorithmic 19 + 19
// populations, 10 + 10 history coefficients and 25 geometry values.
//
// Stencil sites outside a non-periodic face take the linear extrapolation
// 2 j(face) - j(face - normal) per out-of-range axis, filled into the ring
// buffer after the in-domain sites of the plane are known.
#pragma once

#include "lbm_device.cuh"

namespace cslbm {

constexpr int FX = 32, FY = 8, FT = FX * FY;  // interior tile and threads per CTA
constexpr int EX = FX + 2, EY = FY + 2;       // tile with its ring

template <class R> struct FusedSmem {
    R s[2][Q][FY][FX];      // populations (h - w) of the current and the next plane
    R j[3][3][EY][EX];      // rho u of three consecutive planes [slot][component][y][x]
    R geo[NGEO][FY][FX];    // geometry of the plane being stepped (cp.async prefetch)
    R hist[NHIST][FY][FX];  // its forcing history
};

// asynchronous global -> shared copies of one 4- or 8-byte value
template <class R>
__device__ __forceinline__ void cp_async(R* smem, const R* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(R) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ int pslot(int z) { return ((z % 3) + 3) % 3; }

// m1 = sum s c, in the order sums() uses, so both give identical values
template <class R>
__device__ __forceinline__ void sum_m1(const R s[Q], R m1[3])
{
    m1[0] = m1[1] = m1[2] = R(0);
#pragma unroll
    for (int l = 0; l < Q; l++) {
        const int cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
        if (cx) m1[0] += cx * s[l];
        if (cy) m1[1] += cy * s[l];
        if (cz) m1[2] += cz * s[l];
    }
}

// A boundary node of the tile or ring: its populations from the boundary
// rule, rho u into the ring buffer (stride between components js) and, when
// sdst is given, the populations into the plane buffer (stride ss).  Out of
// line so that the common interior path keeps its arrays in registers.
template <class S, class R>
__device__ __noinline__ void boundary_site(const Lat& L, const S* __restrict__ P, const R* __restrict__ hist,
                                           const R* __restrict__ geo, int x, int y, int z, R* jdst, int js, R* sdst,
                                           int ss)
{
    R s[Q], m1[3];
    boundary_pops<S, R>(L, P, hist, geo, x, y, z, s);
    sum_m1(s, m1);
    const long long v = nidx(L, x, y, z);
    const R sg = geo[v];
    for (int a = 0; a < 3; a++) jdst[a * js] = sg * m1[a] + R(0.5) * hist[(1 + a) * L.N + v];
    if (sdst)
        for (int l = 0; l < Q; l++) sdst[l * ss] = s[l];
}

template <class S, class R>
__global__ void __launch_bounds__(FT, sizeof(R) == 4 ? 2 : 1)
    k_step_fused(Lat L, const S* __restrict__ Pin, S* __restrict__ Pout, const R* __restrict__ hin,
                 R* __restrict__ hout, const R* __restrict__ geo, int zc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem<R>& sm = *reinterpret_cast<FusedSmem<R>*>(smem_raw);
    const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
    const long long N = L.N;
    const int tid = threadIdx.x, tx = tid % FX, ty = tid / FX;
    const int ntx = (n0 + FX - 1) / FX;
    const int x0 = (blockIdx.x % ntx) * FX, y0 = (blockIdx.x / ntx) * FY;
    const int w = min(FX, n0 - x0), h = min(FY, n1 - y0);
    const int z0 = blockIdx.y * zc, z1 = min(n2, z0 + zc);
    const bool active = tx < w && ty < h;
    const int x = x0 + tx, y = y0 + ty;
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

    // rho u of plane zz at the tile and ring sites (and the tile's populations);
    // the loads of both sites are issued before either is used
    auto gather_plane = [&](int zz, int buf, bool keep) {
        int zw = zz;
        if (zz < 0 || zz >= n2) {
            if (!zper) return;
            zw = wrapc(zz, n2);
        }
        const int sl = pslot(zz);
        const bool di = active, dr = has_ring && !rghost;
        const bool bi = di && on_boundary(L, x, y, zw), br = dr && on_boundary(L, gx, gy, zw);
        R si[Q], sr[Q];
        const bool fi = di && !bi, fr = dr && !br;
        if (fi) gather_raw<S, R>(L, Pin, x, y, zw, si);
        if (fr) gather_raw<S, R>(L, Pin, gx, gy, zw, sr);
        if (fi) {
            R m1[3];
            sum_m1(si, m1);
            const long long v = nidx(L, x, y, zw);
            const R sg = __ldg(geo + v);
#pragma unroll
            for (int a = 0; a < 3; a++) sm.j[sl][a][ty + 1][tx + 1] = sg * m1[a] + R(0.5) * __ldg(hin + (1 + a) * N + v);
            if (keep)
#pragma unroll
                for (int l = 0; l < Q; l++) sm.s[buf][l][ty][tx] = si[l];
        }
        if (fr) {
            R m1[3];
            sum_m1(sr, m1);
            const long long v = nidx(L, gx, gy, zw);
            const R sg = __ldg(geo + v);
#pragma unroll
            for (int a = 0; a < 3; a++) sm.j[sl][a][ry][rx] = sg * m1[a] + R(0.5) * __ldg(hin + (1 + a) * N + v);
        }
        if (bi)
            boundary_site<S, R>(L, Pin, hin, geo, x, y, zw, &sm.j[sl][0][ty + 1][tx + 1], EY * EX,
                                keep ? &sm.s[buf][0][ty][tx] : nullptr, FY * FX);
        if (br) boundary_site<S, R>(L, Pin, hin, geo, gx, gy, zw, &sm.j[sl][0][ry][rx], EY * EX, nullptr, 0);
    };

    // ring sites outside a non-periodic x or y face of an in-domain plane
    auto fill_xy_ghosts = [&](int zz) {
        if ((zz < 0 || zz >= n2) && !zper) return;
        if (!(has_ring && rghost)) return;
        const int sl = pslot(zz);
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
#pragma unroll
        for (int a = 0; a < 3; a++) {
            R acc = R(0);
            for (int i = 0; i < nx; i++)
                for (int k = 0; k < ny; k++)
                    acc += (i ? R(-1) : (nx == 2 ? R(2) : R(1))) * (k ? R(-1) : (ny == 2 ? R(2) : R(1))) *
                           sm.j[sl][a][k ? cy1 : cy0][i ? cx1 : cx0];
            sm.j[sl][a][ry][rx] = acc;
        }
    };

    // a whole plane one step outside a non-periodic z face
    auto fill_z_ghost = [&](int zz) {
        const int sb = pslot(zz < 0 ? 0 : n2 - 1), si = pslot(zz < 0 ? 1 : n2 - 2), sl = pslot(zz);
        for (int k = tid; k < 3 * EY * EX; k += FT) {
            const int a = k / (EY * EX), r = k % (EY * EX);
            sm.j[sl][a][r / EX][r % EX] = R(2) * sm.j[sb][a][r / EX][r % EX] - sm.j[si][a][r / EX][r % EX];
        }
    };

    gather_plane(z0 - 1, 0, false);
    gather_plane(z0, 0, true);
    __syncthreads();
    fill_xy_ghosts(z0 - 1);
    fill_xy_ghosts(z0);
    __syncthreads();

    for (int z = z0; z < z1; z++) {
        const int cur = (z - z0) & 1;
        // geometry and history of the plane stepped below, copied while the
        // next plane is gathered (each thread reads back only its own node)
        if (active) {
            const long long v = nidx(L, x, y, z);
#pragma unroll
            for (int k = 0; k < NGEO; k++) cp_async(&sm.geo[k][ty][tx], geo + k * N + v);
#pragma unroll
            for (int k = 0; k < NHIST; k++) cp_async(&sm.hist[k][ty][tx], hin + k * N + v);
            cp_async_commit();
        }
        gather_plane(z + 1, cur ^ 1, z + 1 < z1);
        __syncthreads();
        fill_xy_ghosts(z + 1);
        __syncthreads();
        if (!zper && (z == 0 || z == n2 - 1)) {
            if (z == 0) fill_z_ghost(-1);
            if (z == n2 - 1) fill_z_ghost(n2);
            __syncthreads();
        }
        if (active) {
            const long long v = nidx(L, x, y, z);
            cp_async_wait_all();
            Geo<R> G;
            G.sg = sm.geo[0][ty][tx];
            G.isg = R(1) / G.sg;
#pragma unroll
            for (int a = 0; a < 6; a++) G.gi[a] = sm.geo[1 + a][ty][tx];
#pragma unroll
            for (int a = 0; a < 18; a++) G.gam[a] = sm.geo[7 + a][ty][tx];
#pragma unroll
            for (int k = 0; k < 3; k++) G.gc[k] = G.gam[0 * 6 + s6(k, 0)] + G.gam[1 * 6 + s6(k, 1)] + G.gam[2 * 6 + s6(k, 2)];
            Hist<R> Hp;
            Hp.A = sm.hist[0][ty][tx];
#pragma unroll
            for (int a = 0; a < 3; a++) Hp.B[a] = sm.hist[1 + a][ty][tx];
#pragma unroll
            for (int a = 0; a < 6; a++) Hp.C[a] = sm.hist[4 + a][ty][tx];
            R s[Q];
#pragma unroll
            for (int l = 0; l < Q; l++) s[l] = sm.s[cur][l][ty][tx];
            R m0, m1[3], m2[6];
            sums(s, m0, m1, m2);
            const R rho = G.sg * (R(1) + m0) + R(0.5) * Hp.A;
            R j[3];
#pragma unroll
            for (int a = 0; a < 3; a++) j[a] = G.sg * m1[a] + R(0.5) * Hp.B[a];
            R T[6];
            stress(L, G, rho, j, m2, Hp, T);
            // D[k][i] = 1/c_s^2 sum_l w_l c_l^k j^i(x + c_l)  (App. D)
            R D[3][3];
#pragma unroll
            for (int k = 0; k < 3; k++)
#pragma unroll
                for (int i = 0; i < 3; i++) D[k][i] = R(0);
#pragma unroll
            for (int l = 1; l < Q; l++) {
                const int cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
                const R wl = R(3.0 * wq(l));
                const int sl = pslot(z + cz);
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const R jn = sm.j[sl][i][ty + 1 + cy][tx + 1 + cx];
                    if (cx) D[0][i] += (wl * cx) * jn;
                    if (cy) D[1][i] += (wl * cy) * jn;
                    if (cz) D[2][i] += (wl * cz) * jn;
                }
            }
            Hist<R> H;
            forcing_moments(L, G, j, T, D, H);
            store_hist(hout, N, v, H);
            R d0, E1[3], E2[6], trE2;
            collide_coeffs(L, G, m0, rho, j, Hp, H, d0, E1, E2, trE2);
            const R om = R(L.omega);
#pragma unroll
            for (int l = 0; l < Q; l++) {
                const R sn = (R(1) - om) * s[l] + R(wq(l)) * d0 + hermite_l(l, G.isg, R(0), E1, E2, trE2);
                Store<S>::st(Pout + (long long)l * N + v, sn);
            }
        }
        __syncthreads();
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
