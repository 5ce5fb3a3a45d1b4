// Fused LBM step, asynchronously staged form (FP32 storage; n0 a multiple
// of 32, n1 a multiple of 8).
//
// Same method and the same march as k_step_fused (fused_step.cuh): a CTA owns
// a 32 x 8 column, forms rho u of every plane on the tile and a one-node ring
// into a shared-memory ring buffer, and steps the plane below.  The
// difference is how the data arrives.  Every input of a plane is staged in
// shared memory asynchronously, one to two planes ahead of its use:
//   - the pulled populations of destination plane p: for each lambda the
//     12 x 40 box of source rows y0-2..y0+9, columns x0-4..x0+35 of source
//     plane p - c_z, as 16-byte cp.async chunks spread over all threads
//     (periodic edges wrap chunk by chunk); the box covers the tile, its ring
//     and every shift c;
//   - sqrt(g) and B' on the tile and ring of plane p, the same way;
//   - the 25 geometry and 10 history values of the tile of plane p, one 4-D
//     tensor copy each by the copy engine, completion on an mbarrier.
// About 80 KB per plane are in flight while the threads compute, which is
// what keeps HBM busy; the step itself issues no global loads.  The mbarrier
// waits are bounded (half a second): one that runs out raises a flag the host
// reads (CSLBM_ETIMEOUT) and the CTA leaves at the next barrier.
#pragma once

#include <cuda.h>

#include "fused_step.cuh"

namespace cslbm {

namespace tma {

constexpr int TXN = 32, TYN = 8, NT = TXN * TYN;  // tile and threads
constexpr int BX = 40, BY = 12;                   // population box (x0-4.., y0-2..)
constexpr int AX = 40, AY = 10;                   // sqrt(g), B' box (x0-4.., y0-1..)
constexpr int JX = TXN + 2, JY = TYN + 2;         // momentum ring buffer (x0-1.., y0-1..)

struct Smem {
    float pop[3][Q][BY][BX];
    float aux[2][4][AY][AX];
    float geo[2][NGEO][TYN][TXN];
    float hist[2][NHIST][TYN][TXN];
    float4 j[4][JY][JX];
    unsigned long long bar[8];  // geometry/history of the two planes in flight at 5, 6
    int err;
};

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect(unsigned long long* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned long long* b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// bounded wait: false when the phase did not complete within half a second
__device__ __forceinline__ bool bar_wait(unsigned long long* b, unsigned parity)
{
    if (bar_try(b, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (bar_try(b, parity)) return true;
        if (now_ns() - t0 > 500000000ull) return false;
    }
}
__device__ __forceinline__ void tensor4(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                        unsigned long long* b)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(su32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(su32(b))
        : "memory");
}

// c_z of population l for a runtime l
__device__ __forceinline__ int cz_of(int l)
{
    constexpr unsigned plus = (1u << 5) | (1u << 11) | (1u << 14) | (1u << 15) | (1u << 18);
    constexpr unsigned minus = (1u << 6) | (1u << 12) | (1u << 13) | (1u << 16) | (1u << 17);
    return (int)((plus >> l) & 1u) - (int)((minus >> l) & 1u);
}

// A boundary node of the tile: its populations from the boundary rule,
// written into the population box where the pull reads them (each box entry
// (l, x - c_l) is read by this node alone), and rho u into jdst.
__device__ __noinline__ void boundary_into_box(const Lat& L, const float* __restrict__ P, const float* __restrict__ hist,
                                               const float* __restrict__ geo, int x, int y, int z, float* box, int tx,
                                               int ty, float4* jdst)
{
    float s[Q], m1[3];
    boundary_pops<float, float>(L, P, hist, geo, x, y, z, s);
    sum_m1(s, m1);
    const long long v = nidx(L, x, y, z);
    const float sg = geo[v];
    put_j<float>(jdst, sg * m1[0] + 0.5f * hist[1 * L.N + v], sg * m1[1] + 0.5f * hist[2 * L.N + v],
                 sg * m1[2] + 0.5f * hist[3 * L.N + v]);
#pragma unroll
    for (int l = 0; l < Q; l++) box[(l * BY + ty + 2 - cvec(l, 1)) * BX + tx + 4 - cvec(l, 0)] = s[l];
}

}  // namespace tma

__global__ void __launch_bounds__(tma::NT, 1)
    k_step_tma(Lat L, const float* __restrict__ Pin, float* __restrict__ Pout, const float* __restrict__ hin,
               float* __restrict__ hout, const float* __restrict__ geo, int zc,
               const __grid_constant__ CUtensorMap tm_geo, const __grid_constant__ CUtensorMap tm_hist, int* err)
{
    using namespace tma;
    extern __shared__ __align__(128) unsigned char smem_tma[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_tma);
    const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
    const unsigned N = (unsigned)L.N, n01 = (unsigned)n0 * n1;
    const int tid = threadIdx.x, tx = tid % TXN, ty = tid / TXN;
    const int ntx = n0 / TXN;
    const int x0 = (blockIdx.x % ntx) * TXN, y0 = (blockIdx.x / ntx) * TYN;
    const int z0 = blockIdx.y * zc, z1 = min(n2, z0 + zc);
    const int x = x0 + tx, y = y0 + ty;
    const bool xper = L.bclo[0] == BC_PERIODIC, yper = L.bclo[1] == BC_PERIODIC, zper = L.bclo[2] == BC_PERIODIC;

    // ring site of this thread (84 sites): bottom row, top row, left, right
    const int nring = 2 * (TXN + 2) + 2 * TYN;
    int rx, ry;
    if (tid < TXN + 2) { rx = tid; ry = 0; }
    else if (tid < 2 * (TXN + 2)) { rx = tid - (TXN + 2); ry = TYN + 1; }
    else if (tid < 2 * (TXN + 2) + TYN) { rx = 0; ry = tid - 2 * (TXN + 2) + 1; }
    else { rx = TXN + 1; ry = tid - 2 * (TXN + 2) - TYN + 1; }
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
    auto pslot = [](int p) { return ((p % 3) + 3) % 3; };

    if (tid == 0) {
        for (int k = 0; k < 7; k++) bar_init(&sm.bar[k], 1);
        sm.err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    // ---- producers ----------------------------------------------------------
    // The population box of destination plane p holds, for each lambda, the
    // source rows y0-2..y0+9, columns x0-4..x0+35 of source plane p - c_z.
    // Thread t < 228 owns row t of it (lambda = t / 12, row t % 12) for the
    // whole march and copies its ten 16-byte chunks per plane; only the two
    // end chunks can cross a face (periodic: wrapped; otherwise skipped, as
    // only ghost and boundary sites would read them).  Threads t < 40 also
    // own one row of the sqrt(g), B' box (component t / 10, row t % 10).
    const int sx_first = x0 - 4 < 0 ? (xper ? n0 - 4 : -1) : x0 - 4;
    const int sx_last = x0 + TXN >= n0 ? (xper ? 0 : -1) : x0 + TXN;
    const bool has_prow = tid < Q * BY;
    const int pl = has_prow ? tid / BY : 0, pr = tid % BY, pcz = cz_of(pl);
    int psy = y0 - 2 + pr;
    bool pyok = has_prow;
    if (psy < 0 || psy >= n1) {
        if (yper) psy = wrapc(psy, n1);
        else pyok = false;
    }
    const size_t psrc = (size_t)pl * N + (size_t)psy * n0;
    const bool has_arow = tid < 4 * AY;
    const int ak = has_arow ? tid / AY : 0, ar = tid % AY;
    int asy = y0 - 1 + ar;
    bool ayok = has_arow;
    if (asy < 0 || asy >= n1) {
        if (yper) asy = wrapc(asy, n1);
        else ayok = false;
    }
    const float* asrc = (ak == 0 ? geo : hin + (size_t)ak * N) + (size_t)asy * n0;

    auto copy_row = [&](float* dst, const float* src) {
        if (sx_first >= 0) cp_async<16>(dst, src + sx_first);
#pragma unroll
        for (int c = 1; c < BX / 4 - 1; c++) cp_async<16>(dst + 4 * c, src + x0 - 4 + 4 * c);
        if (sx_last >= 0) cp_async<16>(dst + BX - 4, src + sx_last);
    };
    auto issue_pop = [&](int p) {
        int sz;
        if (!pyok || !inplane(p - pcz, sz)) return;
        copy_row(&sm.pop[pslot(p)][pl][pr][0], Pin + psrc + (size_t)sz * n01);
    };
    auto issue_aux = [&](int p) {
        int zw;
        if (!ayok || !inplane(p, zw)) return;
        copy_row(&sm.aux[p & 1][ak][ar][0], asrc + (size_t)zw * n01);
    };
    // one cp.async group per plane: populations and aux of plane p
    auto issue_plane = [&](int p, bool pops, bool aux) {
        if (pops) issue_pop(p);
        if (aux) issue_aux(p);
        cp_async_commit();
    };
    // geometry and history of the tile of plane p: two tensor copies (one
    // thread), completion on the plane's mbarrier
    auto issue_geo = [&](int p) {
        if (tid == 0) {
            unsigned long long* b = &sm.bar[5 + (p & 1)];
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            bar_expect(b, 4u * (NGEO + NHIST) * NT);
            tensor4(&sm.geo[p & 1][0][0][0], &tm_geo, x0, y0, p, 0, b);
            tensor4(&sm.hist[p & 1][0][0][0], &tm_hist, x0, y0, p, 0, b);
        }
    };

    // ---- consumer side ----------------------------------------------------
    unsigned gpar = 0;  // phase bit per geometry buffer
    bool ok = true;
    auto wait_bar = [&](int k, unsigned& par, int bit) {
        if (ok && !bar_wait(&sm.bar[k], (par >> bit) & 1u)) ok = false;
        par ^= 1u << bit;
    };

    // rho u of plane p into the ring buffer
    auto momentum_plane = [&](int p) {
        int zw;
        if (!inplane(p, zw)) return;
        const int ps = pslot(p), as = p & 1, sl = p & 3;
        {
            const bool bnd = on_boundary(L, x, y, zw);
            if (bnd) {
                boundary_into_box(L, Pin, hin, geo, x, y, zw, &sm.pop[ps][0][0][0], tx, ty, &sm.j[sl][ty + 1][tx + 1]);
            } else {
                float s[Q], m1[3];
#pragma unroll
                for (int l = 0; l < Q; l++) s[l] = sm.pop[ps][l][ty + 2 - cvec(l, 1)][tx + 4 - cvec(l, 0)];
                sum_m1(s, m1);
                const float sg = sm.aux[as][0][ty + 1][tx + 4];
                put_j<float>(&sm.j[sl][ty + 1][tx + 1], fmaf(sg, m1[0], 0.5f * sm.aux[as][1][ty + 1][tx + 4]),
                             fmaf(sg, m1[1], 0.5f * sm.aux[as][2][ty + 1][tx + 4]),
                             fmaf(sg, m1[2], 0.5f * sm.aux[as][3][ty + 1][tx + 4]));
            }
        }
        if (has_ring && !rghost) {
            if (on_boundary(L, gx, gy, zw)) {
                scalar_site<float, float, float4>(L, Pin, hin, geo, gx, gy, zw, &sm.j[sl][ry][rx], (float*)nullptr, 0);
            } else {
                float s[Q], m1[3];
#pragma unroll
                for (int l = 0; l < Q; l++) s[l] = sm.pop[ps][l][ry + 1 - cvec(l, 1)][rx + 3 - cvec(l, 0)];
                sum_m1(s, m1);
                const float sg = sm.aux[as][0][ry][rx + 3];
                put_j<float>(&sm.j[sl][ry][rx], fmaf(sg, m1[0], 0.5f * sm.aux[as][1][ry][rx + 3]),
                             fmaf(sg, m1[1], 0.5f * sm.aux[as][2][ry][rx + 3]),
                             fmaf(sg, m1[2], 0.5f * sm.aux[as][3][ry][rx + 3]));
            }
        }
    };

    auto fill_xy_ghosts = [&](int zz) {
        int zw;
        if (!inplane(zz, zw)) return;
        if (!(has_ring && rghost)) return;
        const int sl = zz & 3;
        int cx0 = rx, cx1 = rx, cy0 = ry, cy1 = ry, nx = 1, ny = 1;
        if (xout && !xper) {
            nx = 2;
            if (gx < 0) { cx0 = 1; cx1 = 2; }
            else { cx0 = TXN; cx1 = TXN - 1; }
        }
        if (yout && !yper) {
            ny = 2;
            if (gy < 0) { cy0 = 1; cy1 = 2; }
            else { cy0 = TYN; cy1 = TYN - 1; }
        }
        float acc[3] = {0.f, 0.f, 0.f};
        for (int i = 0; i < nx; i++)
            for (int k = 0; k < ny; k++) {
                const float wt = (i ? -1.f : (nx == 2 ? 2.f : 1.f)) * (k ? -1.f : (ny == 2 ? 2.f : 1.f));
                const float4 jv = sm.j[sl][k ? cy1 : cy0][i ? cx1 : cx0];
                acc[0] += wt * jv.x;
                acc[1] += wt * jv.y;
                acc[2] += wt * jv.z;
            }
        put_j<float>(&sm.j[sl][ry][rx], acc[0], acc[1], acc[2]);
    };
    auto fill_z_ghost = [&](int zz) {
        const int sb = (zz < 0 ? 0 : n2 - 1) & 3, si = (zz < 0 ? 1 : n2 - 2) & 3, sl = zz & 3;
        for (int k = tid; k < JY * JX; k += NT) {
            const float4 a = sm.j[sb][k / JX][k % JX], b = sm.j[si][k / JX][k % JX];
            put_j<float>(&sm.j[sl][k / JX][k % JX], 2.f * a.x - b.x, 2.f * a.y - b.y, 2.f * a.z - b.z);
        }
    };
    // all threads leave together after a barrier when a wait ran out
    auto check_exit = [&]() {
        if (!ok) atomicOr(&sm.err, 1);
        __syncthreads();
        return sm.err != 0;
    };

    // prologue: planes z0-1 and z0 (momentum only), then z0+1 and z0+2 in
    // flight; geometry of z0 and z0+1
    issue_geo(z0);
    if (z0 + 1 < z1) issue_geo(z0 + 1);
    issue_plane(z0 - 1, true, true);
    issue_plane(z0, true, true);
    cp_async_wait<0>();
    __syncthreads();
    momentum_plane(z0 - 1);
    momentum_plane(z0);
    __syncthreads();
    issue_plane(z0 + 1, true, true);
    issue_plane(z0 + 2, z0 + 2 <= z1, z0 + 2 <= z1);
    cp_async_wait<1>();
    fill_xy_ghosts(z0 - 1);
    fill_xy_ghosts(z0);
    __syncthreads();

    for (int z = z0; z < z1; z++) {
        momentum_plane(z + 1);
        __syncthreads();
        fill_xy_ghosts(z + 1);
        __syncthreads();
        if (!zper && (z == 0 || z == n2 - 1)) {
            if (z == 0) fill_z_ghost(-1);
            if (z == n2 - 1) fill_z_ghost(n2);
            __syncthreads();
        }
        wait_bar(5 + (z & 1), gpar, z & 1);
        {
            const int ps = pslot(z), gs = z & 1;
            GeoT<float> G;
            G.sg = sm.geo[gs][0][ty][tx];
            G.isg = 1.0f / G.sg;
#pragma unroll
            for (int a = 0; a < 6; a++) G.gi[a] = sm.geo[gs][1 + a][ty][tx];
#pragma unroll
            for (int a = 0; a < 18; a++) G.gam[a] = sm.geo[gs][7 + a][ty][tx];
#pragma unroll
            for (int k = 0; k < 3; k++) G.gc[k] = (G.gam[0 * 6 + s6(k, 0)] + G.gam[1 * 6 + s6(k, 1)]) + G.gam[2 * 6 + s6(k, 2)];
            HistT<float> Hp;
            Hp.A = sm.hist[gs][0][ty][tx];
#pragma unroll
            for (int a = 0; a < 3; a++) Hp.B[a] = sm.hist[gs][1 + a][ty][tx];
#pragma unroll
            for (int a = 0; a < 6; a++) Hp.C[a] = sm.hist[gs][4 + a][ty][tx];
            float s[Q];
#pragma unroll
            for (int l = 0; l < Q; l++) s[l] = sm.pop[ps][l][ty + 2 - cvec(l, 1)][tx + 4 - cvec(l, 0)];
            PairSums<float> Ps;
            pair_sums(s, Ps);
            float m0, m1[3], m2[6];
            all_moments(s, Ps, m0, m1, m2);
            const float rho = fmaf(G.sg, m0 + 1.0f, 0.5f * Hp.A);
            const float ir = 1.0f / rho;
            float j[3];
#pragma unroll
            for (int a = 0; a < 3; a++) j[a] = fmaf(G.sg, m1[a], 0.5f * Hp.B[a]);
            float Tt[6];
            stress_t<float, float>((float)L.theta, (float)L.kvisc, G, rho, ir, j, m2, Hp, Tt);
            float d[9][3];
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const int l = 2 * k + 1, cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
                const float4 pa = sm.j[(z + cz) & 3][ty + 1 + cy][tx + 1 + cx];
                const float4 ma = sm.j[(z - cz) & 3][ty + 1 - cy][tx + 1 - cx];
                d[k][0] = pa.x - ma.x;
                d[k][1] = pa.y - ma.y;
                d[k][2] = pa.z - ma.z;
            }
            float D[3][3];
            gradient_from_pairs(d, D);
            const float fext[3] = {(float)L.fext[0], (float)L.fext[1], (float)L.fext[2]};
            HistT<float> H;
            forcing_t<float, float>((float)L.theta, fext, G, j, Tt, D, H);
            float out[Q];
            collide_t<float, float>((float)L.omega, (float)L.theta, G, s, m0, rho, ir, j, Hp, H, out);
            const unsigned v = n01 * z + (unsigned)n0 * y + x;
            hout[v] = H.A;
#pragma unroll
            for (int a = 0; a < 3; a++) hout[(1 + a) * N + v] = H.B[a];
#pragma unroll
            for (int a = 0; a < 6; a++) hout[(4 + a) * N + v] = H.C[a];
#pragma unroll
            for (int l = 0; l < Q; l++) Pout[(unsigned)l * N + v] = out[l];
        }
        // plane z+2 (in flight since the previous iteration) must have landed
        // for every thread before the barrier; after it the buffers of plane z
        // are free for plane z+3 and for the geometry of z+2
        cp_async_wait<0>();
        if (check_exit()) {
            if (tid == 0) atomicOr(err, 1);
            return;
        }
        if (z + 3 <= z1) issue_plane(z + 3, true, true);
        if (z + 2 < z1) issue_geo(z + 2);
    }
}

}  // namespace cslbm

namespace cslbm {

// chunks of planes per CTA: about six waves of one CTA per SM
static int tma_chunk(const cslbm_ctx* c)
{
    const int ntiles = (c->n[0] / tma::TXN) * (c->n[1] / tma::TYN);
    int nch = (6 * 152 + ntiles / 2) / ntiles;
    if (nch < 1) nch = 1;
    int zc = (c->n[2] + nch - 1) / nch;
    if (zc < 4) zc = 4;
    if (zc > c->n[2]) zc = c->n[2];
    return zc;
}

bool tma_eligible(const cslbm_ctx* c)
{
    return c->use_tma && c->n[0] % tma::TXN == 0 && c->n[1] % tma::TYN == 0;
}

void launch_tma_step(const cslbm_ctx* c, const Lat& L, const float* Pin, float* Pout, const float* hin,
                            float* hout, const float* geo)
{
    const size_t smem = sizeof(tma::Smem);
    cudaFuncSetAttribute(k_step_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int zc = tma_chunk(c);
    dim3 grid((c->n[0] / tma::TXN) * (c->n[1] / tma::TYN), (c->n[2] + zc - 1) / zc);
    k_step_tma<<<grid, tma::NT, smem, c->stream>>>(L, Pin, Pout, hin, hout, geo, zc, c->tm_geo[c->gc],
                                                   c->tm_hist[c->hc], (int*)(c->scratch + 40));
}

}  // namespace cslbm
