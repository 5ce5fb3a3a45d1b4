// One LBM step in one persistent kernel: the momentum field rho u and the
// step of the interior rows, pipelined over the same row tiles.
//
// The step of a tile needs rho u of the rows around it at time t, which
// needs the populations pulled into those rows -- the same populations the
// step of those rows pulls again.  In the two-kernel form (k_momentum_flat,
// then k_step_rows) the populations cross HBM twice per step.  Here every
// CTA walks its tiles t_k = b + k G (G CTAs, one per SM) and at iteration k
//   1. forms rho u of tile t_k (populations, sqrt(g), A and B staged in a
//      one-stage pipeline) into shared memory;
//   2. steps tile t_{k-m}, m iterations behind, exactly as k_step_rows does
//      (two stages).
// Warps: 8 compute warps; a copy warp for the momentum stage; a copy warp
// for the step stages, which before staging a step tile checks with acquire
// loads (one lane per tile) that each of the up to nine momentum tiles
// holding its rho u rows carries this launch's stamp; and a publishing warp,
// which stores each momentum tile from shared memory with one bulk copy,
// waits for its completion and stamps the tile as published (release).  So
// no compute warp fences or waits on another CTA, and a step tile waits only
// for the CTAs that formed its neighbours, never for all of them.  With
// m >= ceil((nyb + 1) / G) + 1 the tiles a step needs were formed at least
// one iteration earlier, and the populations the step reads were pulled
// through L2 a few iterations before: HBM sees them once per step.
//
// rho u of a face node follows from its inner node without the boundary
// rule's populations: a wall or inflow node takes rho_i u_w (the first
// moment of f^eq(rho_i, u_w) plus the non-equilibrium part of the inner
// node, whose first moment vanishes), an outflow node takes j_i.  So the
// momentum of an interior node next to a face also writes its face nodes:
// into the shared tile when they lie in its row, to HBM (with a fence)
// otherwise.
//
// All CTAs must be resident at once (cooperative launch); every wait is
// bounded (half a second, or the limit of the test hook) and reports through
// *err: bit 1 a copy that did not land, 2 a stage wait of the compute warps,
// 8 a copy warp that stopped early, 16 a step tile whose rho u rows were not
// published in time, 32 / 64 the shared rho u tile's hand-over.
#pragma once

#include "row_step.cuh"

namespace cslbm {
namespace rows {

struct FMaps {
    CUtensorMap pop, pop3, jf, jf3, geo, hist, geo1, hist4;  // pop3: three population planes; jf3: three rho u layers
};

// first moment and density of an interior node i with pulled populations s,
// then rho u of the face nodes whose inner node i is
// returns whether it stored to HBM (the caller then fences before publishing)
static __device__ __noinline__ bool face_momentum(const Lat& L, int xi, int yi, int zi, float rho, float j0, float j1,
                                                  float j2, Mom4<float>* __restrict__ jf, Mom4<float>* row)
{
    bool global = false;
    const float j[3] = {j0, j1, j2};
    const int ri[3] = {xi, yi, zi};
    bool lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lo[a] = L.bclo[a] != BC_PERIODIC && ri[a] == 1;
        hi[a] = L.bchi[a] != BC_PERIODIC && ri[a] == L.n[a] - 2;
    }
    if (!(lo[0] || hi[0] || lo[1] || hi[1] || lo[2] || hi[2])) return false;
#pragma unroll
    for (int dx = -1; dx <= 1; dx++)
#pragma unroll
        for (int dy = -1; dy <= 1; dy++)
#pragma unroll
            for (int dz = -1; dz <= 1; dz++) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                const int dd[3] = {dx, dy, dz};
                bool ok = true;
#pragma unroll
                for (int a = 0; a < 3; a++) ok = ok && (dd[a] == 0 || (dd[a] < 0 ? lo[a] : hi[a]));
                if (!ok) continue;
                int w[3] = {xi + dx, yi + dy, zi + dz}, in[3], axis = 0, side = 0;
                const int bc = classify(L, w, axis, side, in);
                Mom4<float> jw;
                jw.w = 0.0f;
                if (bc == BC_OUTFLOW) {
                    jw.x = j[0];
                    jw.y = j[1];
                    jw.z = j[2];
                } else {
                    const double* fv = nullptr;
#pragma unroll
                    for (int k = 0; k < 6; k++)
                        if (k == axis * 2 + side) fv = L.face[k];
                    float u[3] = {0.0f, 0.0f, 0.0f};
                    if (fv) {
                        const long long fn = face_node(L, axis, w);
                        const long long nf = axis == 0 ? (long long)L.n[1] * L.n[2]
                                                       : (axis == 1 ? (long long)L.n[0] * L.n[2]
                                                                    : (long long)L.n[0] * L.n[1]);
#pragma unroll
                        for (int a = 0; a < 3; a++) u[a] = float(fv[a * nf + fn]);
                    }
                    jw.x = rho * u[0];
                    jw.y = rho * u[1];
                    jw.z = rho * u[2];
                }
                if (dy == 0 && dz == 0) {
                    row[w[0]] = jw;  // same row: part of the tile's bulk store
                } else {
                    jf[nidx(L, w[0], w[1], w[2])] = jw;
                    global = true;
                }
            }
    return global;
}

// copies of the momentum stage of tile t: the population boxes (9 grouped
// boxes when a tile is NT nodes, else 19; rows at a periodic y seam),
// sqrt(g), and A, B of the history
template <class S>
__device__ __forceinline__ void issue_mom(const Lat& L, const Plan& pl, const FMaps& M, int t, unsigned char* st,
                                          unsigned long long* bar, const S* __restrict__ Pin, int lane,
                                          unsigned off_sg, unsigned off_h4, unsigned long long keep)
{
    const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
    const unsigned N = (unsigned)L.N;
    const int zt = t / pl.nyb, y0 = pl.y1 + (t - zt * pl.nyb) * pl.TR, z = pl.z0 + zt;
    const int TRe = min(pl.TR, n1 - y0);
    const bool yper = L.bclo[1] == BC_PERIODIC, zper = L.bclo[2] == BC_PERIODIC;
    const unsigned v0 = ((unsigned)z * n1 + y0) * n0;
    const bool seam = yper && (y0 == 0 || y0 + pl.TR >= n1);
    const bool grouped = !seam && pl.TR * n0 == NT;
    const int npop = seam ? Q * TRe : (grouped ? PGROUPS : Q);
    for (int c = lane; c < npop + 2; c += 32) {
        if (c < npop && grouped) {
            const int base = pgroup_base(c), cnt = pgroup_count(c), d = pgroup_dir(c);
            bool in = true;
            const int zs = wrap_or(z - cvec_rt(d, 2), n2, zper, in);
            bar_expect_tx(bar, (unsigned)(cnt * pl.TR * n0 * sizeof(S)));
            tensor4(st + (size_t)base * NT * sizeof(S), cnt == 3 ? &M.pop3 : &M.pop, 0, y0 - cvec_rt(d, 1), zs, base,
                    bar, keep);
            continue;
        }
        if (c < npop) {
            const int l = seam ? c / TRe : c, r = seam ? c - l * TRe : 0, q = pslot_rt(l);
            bool in = true;
            const int zs = wrap_or(z - cvec_rt(l, 2), n2, zper, in);
            if (!seam) {
                const unsigned bytes = (unsigned)(pl.TR * n0 * sizeof(S));
                bar_expect_tx(bar, bytes);
                tensor4(st + (size_t)q * NT * sizeof(S), &M.pop, 0, y0 - cvec_rt(l, 1), zs, q, bar, keep);
                continue;
            }
            const int ys = wrap_or(y0 + r - cvec_rt(l, 1), n1, yper, in);
            if (!in) continue;
            const unsigned bytes = (unsigned)(n0 * sizeof(S));
            bar_expect_tx(bar, bytes);
            bulk_copy(st + (size_t)(q * NT + r * n0) * sizeof(S), Pin + (size_t)q * N + ((unsigned)zs * n1 + ys) * n0,
                      bytes, bar, keep);
        } else if (c == npop) {
            bar_expect_tx(bar, NT * 4u);
            tensor2(st + off_sg, &M.geo1, (int)v0, 0, bar, keep);
        } else {
            bar_expect_tx(bar, 4u * NT * 4u);
            tensor2(st + off_h4, &M.hist4, (int)v0, 0, bar, keep);
        }
    }
}

// the compute warps' momentum of tile t: inputs into registers, the stage
// handed back, rho u of the interior nodes (and of the face nodes they are
// the inner node of) stored
template <class S>
__device__ __forceinline__ void mom_tile(const Lat& L, const Plan& pl, const unsigned char* st, int t, int tid,
                                         unsigned long long* empty, unsigned long long* jfree, unsigned jfree_parity,
                                         bool jwait, unsigned off_sg, unsigned off_h4, Mom4<float>* __restrict__ js,
                                         Mom4<float>* __restrict__ jf, int* err, unsigned long long wait_ns)
{
    const int n0 = L.n[0], n1 = L.n[1];
    const int r = tid / n0, x = tid - r * n0;
    const int xm = x == 0 ? n0 - 1 : x - 1, xp = x == n0 - 1 ? 0 : x + 1;
    const int qb = r * n0, q0 = qb + x, qm = qb + xm, qp = qb + xp;
    const bool xface = L.bclo[0] != BC_PERIODIC && (x == 0 || x == n0 - 1);
    const bool yper = L.bclo[1] == BC_PERIODIC;
    const int zt = t / pl.nyb, y0 = pl.y1 + (t - zt * pl.nyb) * pl.TR, z = pl.z0 + zt;
    const int y = y0 + r;
    const bool active = r < pl.TR && y < n1 && !(xface || (!yper && (y == 0 || y == n1 - 1)));
    float sv[Q], sg = 0.0f, A = 0.0f, B[3] = {0.0f, 0.0f, 0.0f};
    if (active) {
        const S* pop = reinterpret_cast<const S*>(st);
        const float* gs = reinterpret_cast<const float*>(st + off_sg);
        const float* hs = reinterpret_cast<const float*>(st + off_h4);
#pragma unroll
        for (int l = 0; l < Q; l++) {
            const int cx = cvec(l, 0);
            sv[l] = to_f(pop[pslot(l) * NT + (cx == 0 ? q0 : (cx > 0 ? qm : qp))]);
        }
        sg = gs[q0];
        A = hs[q0];
#pragma unroll
        for (int a = 0; a < 3; a++) B[a] = hs[(1 + a) * NT + q0];
    }
    __syncwarp();
    if ((tid & 31) == 0) bar_arrive(empty);
    // the shared rho u tile of two iterations ago must have been read out
    if (jwait && !bar_wait(jfree, jfree_parity, wait_ns)) atomicOr(err, 32);
    bool global = false;
    if (active) {
        PairSums<float> Ps;
        pair_sums(sv, Ps);
        float m1[3];
        first_moment(Ps, m1);
        float m0 = sv[0];
#pragma unroll
        for (int k = 0; k < 9; k++) m0 += Ps.p[k];
        const float rho = fmad(sg, m0 + 1.0f, 0.5f * A);
        float j[3];
#pragma unroll
        for (int a = 0; a < 3; a++) j[a] = fmad(sg, m1[a], 0.5f * B[a]);
        Mom4<float> o;
        o.x = j[0];
        o.y = j[1];
        o.z = j[2];
        o.w = 0.0f;
        js[r * n0 + x] = o;
        const bool near = (L.bclo[0] != BC_PERIODIC && (x == 1 || x == n0 - 2)) ||
                          (L.bclo[1] != BC_PERIODIC && (y == 1 || y == n1 - 2)) ||
                          (L.bclo[2] != BC_PERIODIC && (z == 1 || z == L.n[2] - 2));
        if (near) global = face_momentum(L, x, y, z, rho, j[0], j[1], j[2], jf, js + r * n0);
    }
    if (global) __threadfence();
    // the tile's shared rows go out through the async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Publication stamps: done[t] holds the number of the last fused launch
// (epoch, counted from 1) whose momentum tile t is stored.  The step of tile
// t reads the rho u rows of the tiles (plane zt + dz, row block yb + dy),
// dz, dy in {-1, 0, 1}; dep_tile gives the k-th of them (k = 3 (dz + 1) +
// (dy + 1)), or -1 where that is no tile (a face plane, written by the tiles
// of plane zt; a y block past a non-periodic end; k >= 9).
__device__ __forceinline__ int dep_tile(const Lat& L, const Plan& pl, int t, int k)
{
    if (k >= 9) return -1;
    const int nz = pl.ntiles / pl.nyb;
    const int zt = t / pl.nyb, yb = t - zt * pl.nyb;
    const int z2 = zt + k / 3 - 1;
    int y2 = yb + k % 3 - 1;
    if (z2 < 0 || z2 >= nz) return -1;
    if (y2 < 0 || y2 >= pl.nyb) {
        if (L.bclo[1] != BC_PERIODIC) return -1;
        y2 = y2 < 0 ? y2 + pl.nyb : y2 - pl.nyb;
    }
    return z2 * pl.nyb + y2;
}
__device__ __forceinline__ bool reached(unsigned v, unsigned target) { return (int)(v - target) >= 0; }

constexpr int NTHR_F = NT + 96;  // compute warps + momentum copy warp + step copy warp + publishing warp

template <class S>
__global__ void __launch_bounds__(NTHR_F, 1)
    k_step_fused(const __grid_constant__ Lat L, const __grid_constant__ Plan pl, const __grid_constant__ FMaps M,
                 const S* __restrict__ Pin, S* __restrict__ Pout, float* __restrict__ hout,
                 Mom4<float>* __restrict__ jf, unsigned* __restrict__ done, unsigned epoch, int m, unsigned off_m,
                 unsigned off_sg, unsigned off_h4, unsigned off_js, int* err, unsigned long long wait_ns, int withhold)
{
    extern __shared__ __align__(128) unsigned char smem_fused[];
    unsigned long long* fullS = reinterpret_cast<unsigned long long*>(smem_fused + off_js + 2u * NT * 16u);
    unsigned long long* emptyS = fullS + 2;
    unsigned long long* fullM = fullS + 4;
    unsigned long long* emptyM = fullS + 5;
    unsigned long long* momDone = fullS + 6;  // [2] the compute warps' rho u of a tile in shared memory
    unsigned long long* jsFree = fullS + 8;   // [2] the publishing warp has read it out
    unsigned char* stM = smem_fused + off_m;
    Mom4<float>* js = reinterpret_cast<Mom4<float>*>(smem_fused + off_js);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            bar_init(&fullS[s], 1);
            bar_init(&emptyS[s], NW);
            bar_init(&momDone[s], NW);
            bar_init(&jsFree[s], 1);
        }
        bar_init(fullM, 1);
        bar_init(emptyM, NW);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const int G = gridDim.x, b = blockIdx.x;
    const int K = pl.ntiles > b ? (pl.ntiles - b + G - 1) / G : 0;
    const int n0 = L.n[0], n1 = L.n[1];

    if (warp == NW) {
        // momentum copy warp
        const unsigned long long keep = policy_evict_last();
        int it = 0;
        for (; it < K; it++) {
            if (it >= 1) {
                if (!__all_sync(0xffffffffu, bar_wait(emptyM, (it - 1) & 1, wait_ns))) break;
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            }
            issue_mom<S>(L, pl, M, b + it * G, stM, fullM, Pin, lane, off_sg, off_h4, keep);
            __syncwarp();
            if (lane == 0) bar_arrive(fullM);
        }
        if (it < K && lane == 0) atomicOr(err, 8);
        if (it > 0 && !bar_wait(fullM, (it - 1) & 1, wait_ns) && lane == 0) atomicOr(err, 2);
    } else if (warp == NW + 1) {
        // step copy warp
        const Pol pol = make_pol();
        int ks = 0;
        for (; ks < K; ks++) {
            const int s = ks & 1, t = b + ks * G;
            if (ks >= 2) {
                if (!__all_sync(0xffffffffu, bar_wait(&emptyS[s], ((ks >> 1) - 1) & 1, wait_ns))) break;
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            }
            unsigned char* st = smem_fused + (size_t)s * pl.stage_bytes;
            // the momentum tiles this step reads must be published: lane k
            // waits for neighbour k of the tile to carry this launch's stamp,
            // before any copy of the tile is in flight
            int dep = 1;
            const int dt = dep_tile(L, pl, t, lane);
            if (dt >= 0) {
                const unsigned long long t0 = now_ns();
                while (!reached(ld_acquire(done + dt), epoch))
                    if (now_ns() - t0 > wait_ns) {
                        dep = 0;
                        break;
                    }
            }
            dep = __all_sync(0xffffffffu, dep);
            asm volatile("fence.proxy.async.global;\n" ::: "memory");
            issue_tile<S>(L, pl, &M.pop, &M.pop3, &M.jf, &M.jf3, &M.geo, &M.hist, t, st, &fullS[s], Pin, jf, lane,
                          dep ? (PART_MAIN | PART_JF) : PART_MAIN, pol);
            __syncwarp();
            if (lane == 0) bar_arrive(&fullS[s]);
            if (!dep) {
                // the tile went out without its rho u rows: report, stop issuing
                if (lane == 0) atomicOr(err, 16);
                ks++;
                break;
            }
        }
        if (ks < K && lane == 0) atomicOr(err, 8);
        for (int j = max(0, ks - 2); j < ks; j++)
            if (!bar_wait(&fullS[j & 1], (j >> 1) & 1, wait_ns) && lane == 0) atomicOr(err, 2);
    } else if (warp == NW + 2) {
        // publishing warp: each momentum tile's rows (face rows excepted)
        // from shared memory to HBM, then the count of its iteration; a CTA
        // past its last tile counts the remaining iterations
        const bool yper = L.bclo[1] == BC_PERIODIC;
        const unsigned long long keep = policy_evict_last();
        int it = 0;
        for (; it < K; it++) {
            const int bb = it & 1, t = b + it * G;
            if (!bar_wait(&momDone[bb], (it >> 1) & 1, wait_ns)) {
                if (lane == 0) atomicOr(err, 64);
                break;
            }
            if (lane == 0) {
                const int zt = t / pl.nyb, y0 = pl.y1 + (t - zt * pl.nyb) * pl.TR, z = pl.z0 + zt;
                const int TRe = min(pl.TR, n1 - y0);
                const int ylo = (!yper && y0 == 0) ? 1 : y0;
                const int yhi = (!yper && y0 + TRe - 1 == n1 - 1) ? n1 - 2 : y0 + TRe - 1;
                if (ylo <= yhi) {
                    const unsigned bytes = (unsigned)((yhi - ylo + 1) * n0 * sizeof(Mom4<float>));
                    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;\n" ::"l"(
                                     jf + ((unsigned)z * n1 + ylo) * n0),
                                 "r"(su32(js + bb * NT + (ylo - y0) * n0)), "r"(bytes), "l"(keep)
                                 : "memory");
                    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
                    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
                }
                bar_arrive(&jsFree[bb]);
                asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
                asm volatile("fence.proxy.async.global;\n" ::: "memory");
                if (!(b == 0 && it == withhold)) st_release(done + t, epoch);
            }
            __syncwarp();
        }
    } else {
        // compute warps
        const unsigned long long pol_store = policy_evict_first();
        for (int it = 0; it < K + m; it++) {
            if (it < K) {
                const int bb = it & 1;
                if (!bar_wait(fullM, it & 1, wait_ns)) {
                    atomicOr(err, 4);
                    break;
                }
                mom_tile<S>(L, pl, stM, b + it * G, tid, emptyM, &jsFree[bb], ((it >> 1) - 1) & 1, it >= 2, off_sg,
                            off_h4, js + bb * NT, jf, err, wait_ns);
                __syncwarp();
                if (lane == 0) bar_arrive(&momDone[bb]);
            }
            const int ks = it - m;
            if (ks >= 0) {
                const int s = ks & 1;
                if (!bar_wait(&fullS[s], (ks >> 1) & 1, wait_ns)) {
                    atomicOr(err, 4);
                    break;
                }
                step_tile<S>(L, pl, smem_fused + (size_t)s * pl.stage_bytes, b + ks * G, tid, &emptyS[s], Pout, hout,
                             pol_store);
            }
        }
    }
    __syncthreads();
}

}  // namespace rows

// one time step through the fused pass, then the face nodes.  Returns the
// number of kernels launched (0: the cooperative launch failed).
template <class S>
int launch_fused_step(cslbm_ctx* c, const Lat& L, int pc, int hc, int gc, int* err)
{
    set_smem_optin_once(rows::k_step_fused<S>, c->device);
    cslbm_rows& R = c->rows;
    const rows::Plan& pl = R.plan;
    const S* Pin = (const S*)c->P[pc];
    S* Pout = (S*)c->P[1 - pc];
    const float* hin = (const float*)c->H[hc];
    float* hout = (float*)c->H[1 - hc];
    const float* geo = (const float*)c->G[gc];
    rows::FMaps M;
    M.pop = R.pop[pc];
    M.pop3 = R.pop3[pc];
    M.jf3 = R.jf3;
    M.jf = R.jf;
    M.geo = R.geo[gc];
    M.hist = R.hist[hc];
    M.geo1 = R.geo1[gc];
    M.hist4 = R.hist4[hc];
    unsigned epoch = R.epoch + 1;  // fused launches including this one; the counts wrap with it
    const int G = pl.ntiles < c->n_sm ? pl.ntiles : c->n_sm;
    // lookahead: the momentum tiles a step tile needs lie at most
    // ceil((nyb + 1) / G) iterations ahead on any CTA; two more absorb the
    // publication latency (a sweep of 1, 2, 4, 7 more on GB300 at 256^3 with
    // per-tile stamps: 1.351, 1.178, 1.199, 1.247 ms per step)
    int m = (pl.nyb + 1 + G - 1) / G + 3;
    unsigned off_m = R.off_m, off_sg = R.off_sg, off_h4 = R.off_h4, off_js = R.off_js;
    Mom4<float>* jf = (Mom4<float>*)c->jf;
    unsigned* done = R.done;
    const rows::Plan plv = pl;
    // the test hook of cslbm_test_withhold_publication applies to this launch only
    unsigned long long wait_ns = R.test_wait_ns ? R.test_wait_ns : rows::kWaitNs;
    int withhold = R.test_withhold;
    R.test_wait_ns = 0;
    R.test_withhold = -1;
    void* args[] = {(void*)&L, (void*)&plv, (void*)&M, (void*)&Pin, (void*)&Pout, (void*)&hout, (void*)&jf,
                    (void*)&done, (void*)&epoch, (void*)&m, (void*)&off_m, (void*)&off_sg, (void*)&off_h4,
                    (void*)&off_js, (void*)&err, (void*)&wait_ns, (void*)&withhold};
    if (cudaLaunchCooperativeKernel((const void*)rows::k_step_fused<S>, dim3(G), dim3(rows::NTHR_F), args,
                                    R.fused_bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    R.epoch = epoch;
    return 1 + launch_faces<S, float>(c, L, Pin, Pout, hin, hout, geo, c->stream);
}

}  // namespace cslbm
