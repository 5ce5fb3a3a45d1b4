// LBM step pass with whole lattice rows staged in shared memory by the
// bulk-copy engine (FP32 arithmetic; FP32, FP16 or BF16 storage).
//
// The step of a node reads, besides its own geometry (25 values) and forcing
// history (10), the populations pulled from its neighbours (Eq. streaming)
// and rho u at the 18 stencil sites of the lattice gradient (App. D).  When
// every thread gathers these itself (k_step_flat), a node costs about a
// hundred global loads with their address arithmetic, and too few of them
// are in flight to cover the HBM latency.  Here a persistent CTA per SM
// splits into NT/32 compute warps and one copy warp.  A tile is TR whole
// x-rows of one plane (TR n0 <= NT nodes).  For a tile the copy warp issues
// one bulk copy (cp.async.bulk, completion on the stage's mbarrier) per
//   - population lambda and tile row: the source row (y - c_y, z - c_z) of
//     array lambda.  It holds every value the row pulls in direction lambda,
//     because the periodic wrap in x stays inside the row;
//   - rho u row of the (TR + 2) x 3 rows around the tile (y0-1 .. y0+TR,
//     z-1 .. z+1);
//   - geometry and history component: TR n0 contiguous values;
// into one of STAGES shared-memory stages.  The compute warps step the
// tile of the previous stage from shared memory and store the new
// populations and history straight to HBM.
//
// Nodes on a non-periodic face (boundary rule, ghost stencil) are left to
// k_step_faces, a separate launch at full occupancy over the face nodes only;
// their rows are not staged, and face planes get no tiles.  Every wait on an
// mbarrier is bounded (half a second); one that runs out sets *err (the host
// reports CSLBM_ETIMEOUT) and the CTA leaves after its copies have landed.
#pragma once

#include <mutex>

#include "flat_step.cuh"
#include "rows_plan.h"

namespace cslbm {
namespace rows {

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(unsigned long long* b, unsigned bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(b)) : "memory");
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
__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// false when the phase of the given parity did not complete within limit_ns
__device__ __forceinline__ bool bar_wait(unsigned long long* b, unsigned parity,
                                         unsigned long long limit_ns = kWaitNs)
{
    if (bar_try(b, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (bar_try(b, parity)) return true;
        if (now_ns() - t0 > limit_ns) return false;
    }
}
// global -> shared bulk copy of `bytes` (16-byte aligned, a multiple of 16)
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* b)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(b))
        : "memory");
}

// c^a of population l for a runtime l (bit masks instead of a table, which
// would live in local memory)
__device__ __forceinline__ int cvec_rt(int l, int a)
{
    constexpr unsigned plus[3] = {(1u << 1) | (1u << 7) | (1u << 9) | (1u << 11) | (1u << 13),
                                  (1u << 3) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 17),
                                  (1u << 5) | (1u << 11) | (1u << 14) | (1u << 15) | (1u << 18)};
    constexpr unsigned minus[3] = {(1u << 2) | (1u << 8) | (1u << 10) | (1u << 12) | (1u << 14),
                                   (1u << 4) | (1u << 8) | (1u << 9) | (1u << 16) | (1u << 18),
                                   (1u << 6) | (1u << 12) | (1u << 13) | (1u << 16) | (1u << 17)};
    const unsigned p = a == 0 ? plus[0] : (a == 1 ? plus[1] : plus[2]);
    const unsigned m = a == 0 ? minus[0] : (a == 1 ? minus[1] : minus[2]);
    return (int)((p >> l) & 1u) - (int)((m >> l) & 1u);
}

// tiled tensor copies (box of the map at the given element coordinates;
// elements outside the tensor read as zero)
__device__ __forceinline__ void tensor2(void* dst, const CUtensorMap* map, int c0, int c1, unsigned long long* b)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(su32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(su32(b))
        : "memory");
}
__device__ __forceinline__ void tensor3(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                        unsigned long long* b)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(su32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(su32(b))
        : "memory");
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

// the same copies carrying an L2 eviction policy (createpolicy)
__device__ __forceinline__ void tensor2(void* dst, const CUtensorMap* map, int c0, int c1, unsigned long long* b,
                                        unsigned long long pol)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
        "{%2, %3}], [%4], %5;\n" ::"r"(su32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(su32(b)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void tensor3(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                        unsigned long long* b, unsigned long long pol)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
        "{%2, %3, %4}], [%5], %6;\n" ::"r"(su32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(su32(b)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void tensor4(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                        unsigned long long* b, unsigned long long pol)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
        "{%2, %3, %4, %5}], [%6], %7;\n" ::"r"(su32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(su32(b)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* b,
                                          unsigned long long pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;\n" ::"r"(su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(b)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ unsigned long long policy_evict_unchanged()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_unchanged.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}

// L2 policies of the staged copies: `once` for data whose last read in the
// step this is (populations in the step stage, geometry, history), `keep`
// for data read again later in the step (the momentum stage's populations,
// sqrt(g), A and B), `shared` for rho u, read by the nine tiles around a row
struct Pol {
    unsigned long long once, keep, shared;
};
__device__ __forceinline__ Pol make_pol()
{
    Pol p;
    p.once = policy_evict_first();
    p.keep = policy_evict_last();
    p.shared = policy_evict_unchanged();
    return p;
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ int wrap_or(int r, int n, bool periodic, bool& inside)
{
    if (r >= 0 && r < n) return r;
    inside = periodic;
    return r < 0 ? r + n : r - n;
}

// Tensor maps handed to the pass (grid constants: a copy instruction must
// name a map in parameter, constant or global memory, never a local copy).
struct Maps {
    CUtensorMap pop, pop3, jf, jf3, geo, hist;  // pop3: three population planes; jf3: three rho u layers
};

// the copy warp: stage the rows of tile t into stage `st`, completing on bar.
// Tiles away from the ends of a periodic y axis take one box per group of
// populations that pull from the same row (three planes, or one: 9 boxes)
// when a tile is NT nodes, else one box per population, then one per rho u
// layer, and one each for the geometry and the history (14 copies); the
// first and last tile of a periodic y axis copy row by row, so that the rows
// across the periodic seam come from the other end of the axis.  The number
// of copies, not their bytes, is what the copy engine pays for.
constexpr int PART_MAIN = 1, PART_JF = 2;  // populations + geometry + history / rho u

template <class S>
__device__ __forceinline__ void issue_tile(const Lat& L, const Plan& pl, const CUtensorMap* mpop,
                                           const CUtensorMap* mpop3, const CUtensorMap* mjf,
                                           const CUtensorMap* mjf3, const CUtensorMap* mgeo,
                                           const CUtensorMap* mhist,
                                           int t, unsigned char* st,
                                           unsigned long long* bar, const S* __restrict__ Pin,
                                           const Mom4<float>* __restrict__ jf, int lane, int part, const Pol& pol,
                                           int stride = 32)
{
    const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
    const unsigned N = (unsigned)L.N;
    const int zt = t / pl.nyb, y0 = pl.y1 + (t - zt * pl.nyb) * pl.TR, z = pl.z0 + zt;
    const int TRe = min(pl.TR, n1 - y0);
    const bool yper = L.bclo[1] == BC_PERIODIC, zper = L.bclo[2] == BC_PERIODIC;
    const unsigned v0 = ((unsigned)z * n1 + y0) * n0;
    const bool seam = yper && (y0 == 0 || y0 + pl.TR >= n1);
    const bool grouped = !seam && pl.TR * n0 == NT;
    // the three rho u layers z - 1 .. z + 1 in one box when they are planes of
    // the lattice and the stage holds them without padding
    const bool jf_one = !seam && pl.JS == (pl.TR + 2) * n0 && z >= 1 && z + 1 <= n2 - 1;
    const int npop = seam ? Q * TRe : (grouped ? PGROUPS : Q), njf = seam ? 3 * (TRe + 2) : (jf_one ? 1 : 3);
    const int total = npop + njf + 2;
    for (int c = lane; c < total; c += stride) {
        const bool is_jf = c >= npop && c < npop + njf;
        if (!(part & (is_jf ? PART_JF : PART_MAIN))) continue;
        if (c < npop && grouped) {
            // planes base .. base + cnt - 1 pull from the same row (y0 - c_y, z - c_z)
            const int base = pgroup_base(c), cnt = pgroup_count(c), d = pgroup_dir(c);
            bool in = true;
            const int zs = wrap_or(z - cvec_rt(d, 2), n2, zper, in);
            bar_expect_tx(bar, (unsigned)(cnt * pl.TR * n0 * sizeof(S)));
            tensor4(st + (size_t)base * NT * sizeof(S), cnt == 3 ? mpop3 : mpop, 0, y0 - cvec_rt(d, 1), zs, base, bar,
                    pol.once);
            continue;
        }
        if (c < npop) {
            const int l = seam ? c / TRe : c, r = seam ? c - l * TRe : 0, q = pslot_rt(l);
            bool in = true;
            const int zs = wrap_or(z - cvec_rt(l, 2), n2, zper, in);
            if (!seam) {
                const unsigned bytes = (unsigned)(pl.TR * n0 * sizeof(S));
                bar_expect_tx(bar, bytes);
                tensor4(st + (size_t)q * NT * sizeof(S), mpop, 0, y0 - cvec_rt(l, 1), zs, q, bar, pol.once);
                continue;
            }
            const int y = y0 + r;
            const int ys = wrap_or(y - cvec_rt(l, 1), n1, yper, in);
            if (!in) continue;
            const unsigned bytes = (unsigned)(n0 * sizeof(S));
            bar_expect_tx(bar, bytes);
            bulk_copy(st + (size_t)(q * NT + r * n0) * sizeof(S), Pin + (size_t)q * N + ((unsigned)zs * n1 + ys) * n0,
                      bytes, bar, pol.once);
        } else if (c < npop + njf && jf_one) {
            // rows y0 - 1 .. y0 + TR of planes z - 1 .. z + 1 (row -1 of the first
            // tile is the fill: only face rows use it)
            bar_expect_tx(bar, (unsigned)(3 * (pl.TR + 2) * n0 * sizeof(Mom4<float>)));
            tensor3(st + pl.off_jf, mjf3, 0, (y0 - 1) * 4 * n0 / pl.JL, z - 1, bar, pol.shared);
        } else if (c < npop + njf) {
            const int k = c - npop, a = seam ? k / (TRe + 2) : k, b = seam ? k - a * (TRe + 2) : 0;
            bool in = true;
            const int zs = wrap_or(z - 1 + a, n2, zper, in);
            if (!in) continue;
            unsigned char* dst = st + pl.off_jf + (size_t)(a * pl.JS + b * n0) * sizeof(Mom4<float>);
            if (!seam) {
                const unsigned bytes = (unsigned)((pl.TR + 2) * n0 * sizeof(Mom4<float>));
                bar_expect_tx(bar, bytes);
                // first line of rows y0 - 1 .. y0 + TR of plane zs (row y0 - 1 of
                // the first tile reads the previous plane's last row or the
                // fill: only face rows use it)
                const int line = (int)(((long long)zs * n1 + y0 - 1) * 4 * n0 / pl.JL);
                tensor2(dst, mjf, 0, line, bar, pol.shared);
                continue;
            }
            const int ys = wrap_or(y0 - 1 + b, n1, yper, in);
            if (!in) continue;
            const unsigned bytes = (unsigned)(n0 * sizeof(Mom4<float>));
            bar_expect_tx(bar, bytes);
            bulk_copy(dst, jf + ((unsigned)zs * n1 + ys) * n0, bytes, bar, pol.shared);
        } else if (c == npop + njf) {
            bar_expect_tx(bar, NGEO * NT * 4u);
            tensor2(st + pl.off_geo, mgeo, (int)v0, 0, bar, pol.once);
        } else {
            bar_expect_tx(bar, NHIST * NT * 4u);
            tensor2(st + pl.off_hist, mhist, (int)v0, 0, bar, pol.once);
        }
    }
}

// The compute warps' part of a staged tile: every input of the thread's node
// into registers, the stage handed back to the copy warp (one arrive per
// warp on `empty`), then the step of the node, stored straight to HBM.
// Nodes on a face are left to k_step_faces.
template <class S>
__device__ __forceinline__ void step_tile(const Lat& L, const Plan& pl, const unsigned char* st, int t, int tid,
                                          unsigned long long* empty, S* __restrict__ Pout, float* __restrict__ hout,
                                          unsigned long long pol_store)
{
    const int n0 = L.n[0], n1 = L.n[1];
    const unsigned N = (unsigned)L.N;
    const int r = tid / n0, x = tid - r * n0;
    const int xm = x == 0 ? n0 - 1 : x - 1, xp = x == n0 - 1 ? 0 : x + 1;
    const int qb = r * n0, q0 = qb + x, qm = qb + xm, qp = qb + xp;
    const bool xface = L.bclo[0] != BC_PERIODIC && (x == 0 || x == n0 - 1);
    const bool yper = L.bclo[1] == BC_PERIODIC;
    const int zt = t / pl.nyb, y0 = pl.y1 + (t - zt * pl.nyb) * pl.TR, z = pl.z0 + zt;
    const int y = y0 + r;
    // nodes on a face are stepped by k_step_faces
    const bool active = r < pl.TR && y < n1 && !(xface || (!yper && (y == 0 || y == n1 - 1)));
    // every input of the node into registers first, so that the stage
    // goes back to the copy warp before the arithmetic starts
    float sv[Q];
    GeoT<float> G;
    HistT<float> Hp;
    float d[9][3];
    if (active) {
        const S* pop = reinterpret_cast<const S*>(st);
        const float* gs = reinterpret_cast<const float*>(st + pl.off_geo);
        const float* hs = reinterpret_cast<const float*>(st + pl.off_hist);
        const Mom4<float>* js = reinterpret_cast<const Mom4<float>*>(st + pl.off_jf);
#pragma unroll
        for (int l = 0; l < Q; l++) {
            const int cx = cvec(l, 0);
            sv[l] = to_f(pop[pslot(l) * NT + (cx == 0 ? q0 : (cx > 0 ? qm : qp))]);
        }
        G.sg = gs[q0];
#pragma unroll
        for (int a = 0; a < 6; a++) G.gi[a] = gs[(1 + a) * NT + q0];
#pragma unroll
        for (int a = 0; a < 18; a++) G.gam[a] = gs[(7 + a) * NT + q0];
        Hp.A = hs[q0];
#pragma unroll
        for (int a = 0; a < 3; a++) Hp.B[a] = hs[(1 + a) * NT + q0];
#pragma unroll
        for (int a = 0; a < 6; a++) Hp.C[a] = hs[(4 + a) * NT + q0];
        // rho u at site (x + cx, y + cy, z + cz): layer cz + 1, row r + 1 + cy
        const int jb = n0;  // row r + 1 starts at (r + 1) n0 = qb + n0
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const int l = 2 * k + 1, cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
            const int ip = (cz + 1) * pl.JS + cy * jb + jb + (cx == 0 ? q0 : (cx > 0 ? qp : qm));
            const int im = (1 - cz) * pl.JS - cy * jb + jb + (cx == 0 ? q0 : (cx > 0 ? qm : qp));
            const Mom4<float> p = js[ip], m = js[im];
            d[k][0] = p.x - m.x;
            d[k][1] = p.y - m.y;
            d[k][2] = p.z - m.z;
        }
    }
    __syncwarp();
    if ((tid & 31) == 0) bar_arrive(empty);
    if (active) {
        G.isg = recip(G.sg);
#pragma unroll
        for (int k = 0; k < 3; k++)
            G.gc[k] = (G.gam[0 * 6 + s6(k, 0)] + G.gam[1 * 6 + s6(k, 1)]) + G.gam[2 * 6 + s6(k, 2)];
        const unsigned v = ((unsigned)z * n1 + y) * n0 + x;
        step_core<S, float, true>(L, sv, G, Hp, d, Pout, hout, v, N, pol_store);
    }
}

template <class S>
__global__ void __launch_bounds__(NTHR, 1)
    k_step_rows(const __grid_constant__ Lat L, const __grid_constant__ Plan pl, const __grid_constant__ Maps M,
                const S* __restrict__ Pin, S* __restrict__ Pout, float* __restrict__ hout,
                const Mom4<float>* __restrict__ jf, int* err)
{
    extern __shared__ __align__(128) unsigned char smem_rows[];
    unsigned long long* full = reinterpret_cast<unsigned long long*>(smem_rows + STAGES * pl.stage_bytes);
    unsigned long long* empty = full + STAGES;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const int n0 = L.n[0], n1 = L.n[1];

    if (tid >= NT) {
        // copy warp
        const int lane = tid - NT;
        const Pol pol = make_pol();
        int i = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < pl.ntiles; t += gridDim.x, i++) {
            const int s = i % STAGES;
            if (i >= STAGES) {
                ok = bar_wait(&empty[s], ((i / STAGES) - 1) & 1);
                if (!__all_sync(0xffffffffu, ok)) break;
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            }
            issue_tile<S>(L, pl, &M.pop, &M.pop3, &M.jf, &M.jf3, &M.geo, &M.hist, t, smem_rows + (size_t)s * pl.stage_bytes,
                          &full[s], Pin, jf, lane, PART_MAIN | PART_JF, pol);
            __syncwarp();
            if (lane == 0) bar_arrive(&full[s]);
        }
        if (!ok && lane == 0) atomicOr(err, 1);
        // leave only when the copies of the last stages have landed
        for (int j = max(0, i - STAGES); j < i; j++)
            if (!bar_wait(&full[j % STAGES], (j / STAGES) & 1) && lane == 0) atomicOr(err, 2);
    } else {
        // compute warps
        const unsigned long long pol_store = policy_evict_first();
        int i = 0;
        for (int t = blockIdx.x; t < pl.ntiles; t += gridDim.x, i++) {
            const int s = i % STAGES;
            if (!bar_wait(&full[s], (i / STAGES) & 1)) {
                atomicOr(err, 4);
                break;
            }
            step_tile<S>(L, pl, smem_rows + (size_t)s * pl.stage_bytes, t, tid, &empty[s], Pout, hout, pol_store);
        }
    }
    __syncthreads();
}

}  // namespace rows

// The opt-in shared-memory limit of a kernel, set once per device: the
// attribute belongs to the context of the device current when it is set.
template <class K>
inline void set_smem_optin_once(K* kernel, int device)
{
    static std::mutex mu;
    static bool done[64] = {};
    if (device < 0 || device >= 64) return;
    std::lock_guard<std::mutex> lock(mu);
    if (done[device]) return;
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    done[device] = true;
}

// one time step through the row-staged pass (the context's plan and maps
// exist): momentum pass, row pass, face nodes.  Returns the number of
// kernels launched.
template <class S>
int launch_rows_step(const cslbm_ctx* c, const Lat& L, int pc, int hc, int gc, int* err)
{
    set_smem_optin_once(rows::k_step_rows<S>, c->device);
    const cslbm_rows& R = c->rows;
    const rows::Plan& pl = R.plan;
    const S* Pin = (const S*)c->P[pc];
    S* Pout = (S*)c->P[1 - pc];
    const float* hin = (const float*)c->H[hc];
    float* hout = (float*)c->H[1 - hc];
    const float* geo = (const float*)c->G[gc];
    launch_momentum<S, float>(c, L, Pin, hin, geo);
    int launched = 1;
    if (pl.ntiles > 0) {
        rows::Maps M;
        M.pop = R.pop[pc];
        M.pop3 = R.pop3[pc];
        M.jf3 = R.jf3;
        M.jf = R.jf;
        M.geo = R.geo[gc];
        M.hist = R.hist[hc];
        const int grid = pl.ntiles < c->n_sm ? pl.ntiles : c->n_sm;
        rows::k_step_rows<S><<<grid, rows::NTHR, rows::smem_bytes(pl), c->stream>>>(L, pl, M, Pin, Pout, hout,
                                                                                   (const Mom4<float>*)c->jf, err);
        launched++;
    }
    launched += launch_faces<S, float>(c, L, Pin, Pout, hin, hout, geo, c->stream);
    return launched;
}

}  // namespace cslbm
