// Batched form: many independent channels of uneven sizes advanced together,
// FP32 storage.
//
// Each channel is an ordinary context (its own workspace slice, metric,
// boundary velocities; every single-channel call works on it).  A time step
// of the whole batch is ONE persistent launch: a grid of CTAs, all resident
// at once (cooperative launch), takes work items -- runs of `item` nodes of
// one channel -- from a device-side queue (an atomic counter over the items
// of every channel laid end to end), forms the momentum field rho u of each
// (the gather pass's per-node code), meets at a grid barrier, then takes the
// step items from a second queue (pull, moments, gradient, forcing,
// collision, store).  A CTA finds an item's channel by binary search in the
// channels' first items, held in shared memory; the channel's lattice,
// buffers and ping-pong parities come from a table in device memory.  The
// queue lets small and large channels share the SMs without a fixed block
// assignment.  Two steps are captured once as a CUDA graph (queue reset,
// launch, queue reset, launch) on the batch's own stream and replayed; the
// table is re-uploaded only when a channel's buffers moved (a metric update,
// a single-channel step).  The tile shape -- nodes per block, nodes per work
// item, blocks per SM -- is picked by cslbm_batch_tune, which times every
// candidate on the batch itself with the same step repeated from the same
// input (the state does not advance).  The grid barrier's wait is bounded
// (half a second); a wait that runs out sets the batch's error flag, which
// cslbm_batch_check reports as CSLBM_ETIMEOUT.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "ctx.h"
#include "make_lat.h"
#include "flat_step.cuh"

namespace cslbm {
namespace batch {

struct Chan {
    Lat L;
    float* P[2];
    float* H[2];
    const float* G;
    Mom4<float>* jf;
    int pc0, hc0;  // the context's buffers when the table was made
};

constexpr int kMaxChan = 4096;

__device__ __forceinline__ int find_chan(const unsigned* blk0, int nchan, unsigned blk)
{
    int lo = 0, hi = nchan - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk0[mid] <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr unsigned long long kWaitNs = 500000000ull;
constexpr int kTB[3] = {128, 256, 512};       // nodes per block
constexpr int kItemMul[3] = {1, 4, 16};       // nodes per work item, in blocks
constexpr int kItems[7] = {128, 256, 512, 1024, 2048, 4096, 8192};

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// every CTA of the grid here before any goes on (bounded; *err |= 1 when
// the wait ran out): the momentum field is complete for the step phase
__device__ __forceinline__ void grid_barrier(unsigned* count, int* err)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        const unsigned long long t0 = now_ns();
        unsigned v;
        for (;;) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(count) : "memory");
            if (v >= gridDim.x) break;
            if (now_ns() - t0 > kWaitNs) {
                atomicOr(err, 1);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// One persistent launch per LBM step of every channel (see the top of the
// file).  first[c] = first work item of channel c (items of `item` nodes),
// first[nchan] = all items; q[0], q[1] the momentum and step queues and
// q[2] the barrier count, zero at launch; k the parity of the step in the
// two-step cycle.
template <int TB>
__global__ void __launch_bounds__(TB) k_batch_persistent(const Chan* __restrict__ tab,
                                                         const unsigned* __restrict__ first, int nchan, int item,
                                                         int k, unsigned* q, int* err)
{
    extern __shared__ unsigned sb[];
    __shared__ unsigned w_s;
    for (int i = threadIdx.x; i <= nchan; i += TB) sb[i] = first[i];
    __syncthreads();
    const unsigned nitems = sb[nchan];
    for (int phase = 0; phase < 2; phase++) {
        for (;;) {
            if (threadIdx.x == 0) w_s = atomicAdd(&q[phase], 1u);
            __syncthreads();
            const unsigned w = w_s;
            __syncthreads();
            if (w >= nitems) break;
            const int c = find_chan(sb, nchan, w);
            const Chan& C = tab[c];
            const unsigned N = (unsigned)C.L.N, v0 = (w - sb[c]) * (unsigned)item;
            const unsigned v1 = min(v0 + (unsigned)item, N);
            const unsigned n0 = C.L.n[0], n01 = n0 * C.L.n[1];
            const int pi = (C.pc0 + k) & 1, hi = (C.hc0 + k) & 1;
            for (unsigned v = v0 + threadIdx.x; v < v1; v += TB) {
                const int z = (int)(v / n01), r = (int)(v - z * n01), y = r / (int)n0, x = r - y * (int)n0;
                if (phase == 0)
                    momentum_node<float, float>(C.L, C.P[pi], C.H[hi], C.G, C.jf, x, y, z, v);
                else
                    step_node<float, float>(C.L, C.P[pi], C.P[pi ^ 1], C.H[hi], C.H[hi ^ 1], C.G, C.jf, x, y, z, v);
            }
        }
        if (phase == 0) grid_barrier(&q[2], err);
    }
}

}  // namespace batch
}  // namespace cslbm

using cslbm::batch::Chan;

struct Shape {
    int tb;    // index into kTB
    int item;  // nodes per work item
    int bps;   // blocks per SM
};

struct cslbm_batch {
    int nb;
    std::vector<cslbm_ctx*> ctx;
    cudaStream_t user;    // the caller's stream
    cudaStream_t stream;  // the batch's own stream (graphs are captured on it)
    cudaEvent_t ev_in, ev_out, t0, t1;
    Chan* d_tab;          // [nb] in the workspace
    unsigned* d_first;    // [7][nb + 1]: first work item of each channel, per item size of kItems
    unsigned* d_q;        // [4]: momentum queue, step queue, barrier count, unused
    int* d_err;           // grid-barrier timeout flag
    std::vector<Chan> h_tab;
    std::vector<unsigned> h_first;
    int n_sm;
    Shape shape;
    std::vector<Shape> cand;  // the tuner's candidates, and their times
    std::vector<float> cand_ms;
    cudaGraphExec_t graph;    // two steps
    Shape graph_shape;
    int have_table;
    long long launches;
};

namespace {

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

cslbm_status bfail(cslbm_status s, const std::string& m) { return cslbm_record_error(s, m.c_str()); }

#define BCUDA(x)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (x);                                                                             \
        if (e_ != cudaSuccess) return bfail(CSLBM_ECUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
    } while (0)

bool same(const Shape& a, const Shape& b) { return a.tb == b.tb && a.item == b.item && a.bps == b.bps; }

int item_index(int item)
{
    for (int i = 0; i < 7; i++)
        if (cslbm::batch::kItems[i] == item) return i;
    return 0;
}

bool table_current(const cslbm_batch* b)
{
    if (!b->have_table) return false;
    for (int i = 0; i < b->nb; i++) {
        const cslbm_ctx* c = b->ctx[i];
        const Chan& t = b->h_tab[i];
        if (t.pc0 != c->pc || t.hc0 != c->hc || t.G != (const float*)c->G[c->gc]) return false;
    }
    return true;
}

cslbm_status upload_table(cslbm_batch* b)
{
    for (int i = 0; i < b->nb; i++) {
        const cslbm_ctx* c = b->ctx[i];
        Chan& t = b->h_tab[i];
        t.L = cslbm::make_lat(c);
        for (int k = 0; k < 2; k++) {
            t.P[k] = (float*)c->P[k];
            t.H[k] = (float*)c->H[k];
        }
        t.G = (const float*)c->G[c->gc];
        t.jf = (cslbm::Mom4<float>*)c->jf;
        t.pc0 = c->pc;
        t.hc0 = c->hc;
    }
    BCUDA(cudaMemcpyAsync(b->d_tab, b->h_tab.data(), b->nb * sizeof(Chan), cudaMemcpyHostToDevice, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    b->have_table = 1;
    return CSLBM_OK;
}

template <int TB>
cudaError_t launch_tb(cslbm_batch* b, const Shape& sh, int k, cudaStream_t s)
{
    const unsigned* first = b->d_first + item_index(sh.item) * (b->nb + 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sh.bps * b->n_sm));
    cfg.blockDim = dim3(TB);
    cfg.dynamicSmemBytes = (b->nb + 1) * sizeof(unsigned);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cslbm::batch::k_batch_persistent<TB>, (const Chan*)b->d_tab, first, b->nb,
                              sh.item, k, b->d_q, b->d_err);
}

// one LBM step of every channel: the queues reset, then one persistent launch
cudaError_t launch_step(cslbm_batch* b, const Shape& sh, int k, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(b->d_q, 0, 4 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    switch (sh.tb) {
    case 0: return launch_tb<128>(b, sh, k, s);
    case 1: return launch_tb<256>(b, sh, k, s);
    default: return launch_tb<512>(b, sh, k, s);
    }
}

int occupancy(const cslbm_batch* b, int tb)
{
    int occ = 0;
    const size_t sm = (b->nb + 1) * sizeof(unsigned);
    switch (tb) {
    case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cslbm::batch::k_batch_persistent<128>, 128, sm); break;
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cslbm::batch::k_batch_persistent<256>, 256, sm); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cslbm::batch::k_batch_persistent<512>, 512, sm); break;
    }
    return occ;
}

cslbm_status make_graph(cslbm_batch* b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t g;
    BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e0 = launch_step(b, b->shape, 0, b->stream);
    cudaError_t e1 = e0 == cudaSuccess ? launch_step(b, b->shape, 1, b->stream) : e0;
    cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
    if (e1 != cudaSuccess || ec != cudaSuccess)
        return bfail(CSLBM_ECUDA, std::string("batch step capture: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : ec));
    cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(CSLBM_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
    b->graph_shape = b->shape;
    return CSLBM_OK;
}

}  // namespace

extern "C" {

cslbm_status cslbm_batch_workspace_bytes(int nb, const cslbm_params* p, size_t* bytes)
{
    if (nb <= 0 || nb > cslbm::batch::kMaxChan || !p || !bytes) return bfail(CSLBM_EINVAL, "bad argument");
    size_t total = 0;
    for (int i = 0; i < nb; i++) {
        if (p[i].storage != CSLBM_FP32) return bfail(CSLBM_EINVAL, "a batch holds FP32 channels only");
        size_t w = 0;
        if (cslbm_status s = cslbm_workspace_bytes(&p[i], &w)) return s;
        total += al(w);
    }
    total += al(nb * sizeof(Chan)) + al(7 * (nb + 1) * sizeof(unsigned)) + al(4 * sizeof(unsigned) + sizeof(int));
    *bytes = total;
    return CSLBM_OK;
}

cslbm_status cslbm_batch_create(int nb, const cslbm_params* p, void* workspace, size_t bytes, void* stream,
                                cslbm_batch** out)
{
    if (!out || !workspace) return bfail(CSLBM_EINVAL, "null argument");
    size_t need = 0;
    if (cslbm_status s = cslbm_batch_workspace_bytes(nb, p, &need)) return s;
    if (bytes < need) return bfail(CSLBM_ENOMEM, "workspace smaller than cslbm_batch_workspace_bytes");
    if ((uintptr_t)workspace & 255) return bfail(CSLBM_EINVAL, "workspace must be 256-byte aligned");
    cslbm_batch* b = new cslbm_batch();
    b->nb = nb;
    b->user = (cudaStream_t)stream;
    b->graph = nullptr;
    b->graph_shape = {-1, 0, 0};
    b->have_table = 0;
    b->launches = 0;
    char* base = (char*)workspace;
    size_t o = 0;
    cslbm_status st = CSLBM_OK;
    for (int i = 0; i < nb && !st; i++) {
        size_t w = 0;
        cslbm_workspace_bytes(&p[i], &w);
        cslbm_params q = p[i];
        q.step_kernel = CSLBM_STEP_FLAT;  // a channel's own steps take the same gather pass
        cslbm_ctx* c = nullptr;
        st = cslbm_create(&q, base + o, w, stream, &c);
        if (!st) b->ctx.push_back(c);
        o += al(w);
    }
    b->d_tab = (Chan*)(base + o);
    o += al(nb * sizeof(Chan));
    b->d_first = (unsigned*)(base + o);
    o += al(7 * (nb + 1) * sizeof(unsigned));
    b->d_q = (unsigned*)(base + o);
    b->d_err = (int*)(b->d_q + 4);
    b->h_tab.resize(nb);
    b->h_first.assign(7 * (nb + 1), 0);
    for (int t = 0; t < 7 && !st; t++) {
        unsigned acc = 0;
        for (int i = 0; i < nb; i++) {
            b->h_first[t * (nb + 1) + i] = acc;
            acc += (unsigned)((b->ctx[i]->N + cslbm::batch::kItems[t] - 1) / cslbm::batch::kItems[t]);
        }
        b->h_first[t * (nb + 1) + nb] = acc;
    }
    bool have_stream = false;
    if (!st) {
        cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->ctx[0]->device);
        b->shape = {1, 1024, 1};
        const int occ = occupancy(b, 1);
        if (occ < 1) st = bfail(CSLBM_ECUDA, "the batch kernel cannot be resident");
        else b->shape.bps = occ;
    }
    if (!st) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            st = bfail(CSLBM_ECUDA, "stream creation failed");
        else
            have_stream = true;
    }
    if (!st && (cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess))
        st = bfail(CSLBM_ECUDA, "event creation failed");
    if (!st && cudaMemcpyAsync(b->d_first, b->h_first.data(), 7 * (nb + 1) * sizeof(unsigned), cudaMemcpyHostToDevice,
                               b->stream) != cudaSuccess)
        st = bfail(CSLBM_ECUDA, "table upload failed");
    if (!st && cudaMemsetAsync(b->d_q, 0, 4 * sizeof(unsigned) + sizeof(int), b->stream) != cudaSuccess)
        st = bfail(CSLBM_ECUDA, "queue reset failed");
    if (!st && cudaStreamSynchronize(b->stream) != cudaSuccess) st = bfail(CSLBM_ECUDA, "table upload failed");
    if (st) {
        if (have_stream) cudaStreamDestroy(b->stream);
        for (cslbm_ctx* c : b->ctx) cslbm_destroy(c);
        delete b;
        return st;
    }
    *out = b;
    return CSLBM_OK;
}

cslbm_status cslbm_batch_context(cslbm_batch* b, int i, cslbm_ctx** out)
{
    if (!b || !out || i < 0 || i >= b->nb) return bfail(CSLBM_EINVAL, "bad argument");
    *out = b->ctx[i];
    return CSLBM_OK;
}

cslbm_status cslbm_batch_step(cslbm_batch* b, int nsteps)
{
    if (!b || nsteps < 0) return bfail(CSLBM_EINVAL, "bad argument");
    for (cslbm_ctx* c : b->ctx)
        if (!c->has_state) return bfail(CSLBM_ESTATE, "a channel of the batch has no state");
    if (nsteps == 0) return CSLBM_OK;
    // the batch stream starts after the caller's queued work
    BCUDA(cudaEventRecord(b->ev_in, b->user));
    BCUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    if (!table_current(b))
        if (cslbm_status s = upload_table(b)) return s;
    if (!b->graph || !same(b->graph_shape, b->shape))
        if (cslbm_status s = make_graph(b)) return s;
    for (int t = 0; t + 1 < nsteps; t += 2) {
        BCUDA(cudaGraphLaunch(b->graph, b->stream));
        b->launches += 2;
    }
    if (nsteps & 1) {
        BCUDA(launch_step(b, b->shape, 0, b->stream));
        b->launches += 1;
    }
    for (cslbm_ctx* c : b->ctx) {
        c->pc ^= nsteps & 1;
        c->hc ^= nsteps & 1;
    }
    // the caller's stream waits for the batch
    BCUDA(cudaEventRecord(b->ev_out, b->stream));
    BCUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return CSLBM_OK;
}

cslbm_status cslbm_batch_tune(cslbm_batch* b, int reps, int* shape3, float* ms)
{
    if (!b || reps <= 0) return bfail(CSLBM_EINVAL, "bad argument");
    for (cslbm_ctx* c : b->ctx)
        if (!c->has_state) return bfail(CSLBM_ESTATE, "a channel of the batch has no state");
    BCUDA(cudaEventRecord(b->ev_in, b->user));
    BCUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    if (!table_current(b))
        if (cslbm_status s = upload_table(b)) return s;
    // candidates: block size x work-item size x blocks per SM (the resident
    // maximum and half of it); the same step (parity 0) repeated, so every
    // repetition reads the current state and writes the spare buffers
    b->cand.clear();
    b->cand_ms.clear();
    for (int t = 0; t < 3; t++) {
        const int occ = occupancy(b, t);
        if (occ < 1) continue;
        const int bps_c[2] = {occ, occ / 2};
        for (int u = 0; u < 2; u++) {
            if (bps_c[u] < 1 || (u == 1 && bps_c[1] == bps_c[0])) continue;
            for (int mi = 0; mi < 3; mi++) b->cand.push_back({t, cslbm::batch::kTB[t] * cslbm::batch::kItemMul[mi], bps_c[u]});
        }
    }
    float best = 1e30f;
    Shape best_s = b->shape;
    for (const Shape& sh : b->cand) {
        BCUDA(launch_step(b, sh, 0, b->stream));  // warm
        BCUDA(cudaEventRecord(b->t0, b->stream));
        for (int r = 0; r < reps; r++) BCUDA(launch_step(b, sh, 0, b->stream));
        BCUDA(cudaEventRecord(b->t1, b->stream));
        BCUDA(cudaEventSynchronize(b->t1));
        float e = 0.0f;
        BCUDA(cudaEventElapsedTime(&e, b->t0, b->t1));
        b->cand_ms.push_back(e / reps);
        if (e < best) {
            best = e;
            best_s = sh;
        }
    }
    b->shape = best_s;
    if (shape3) {
        shape3[0] = cslbm::batch::kTB[best_s.tb];
        shape3[1] = best_s.item;
        shape3[2] = best_s.bps;
    }
    if (ms) *ms = best / reps;
    BCUDA(cudaEventRecord(b->ev_out, b->stream));
    BCUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return CSLBM_OK;
}

cslbm_status cslbm_batch_set_shape(cslbm_batch* b, const int* shape3)
{
    if (!b || !shape3) return bfail(CSLBM_EINVAL, "bad argument");
    int t = -1;
    for (int k = 0; k < 3; k++)
        if (cslbm::batch::kTB[k] == shape3[0]) t = k;
    bool item_ok = false;
    for (int k = 0; k < 7; k++)
        if (cslbm::batch::kItems[k] == shape3[1]) item_ok = true;
    if (t < 0 || !item_ok || shape3[1] % shape3[0] != 0 || shape3[2] < 1 || shape3[2] > occupancy(b, t))
        return bfail(CSLBM_EINVAL, "nodes per block 128, 256 or 512; nodes per work item a multiple of it in "
                                   "128..8192 (powers of two); blocks per SM from 1 to the resident maximum");
    b->shape = {t, shape3[1], shape3[2]};
    return CSLBM_OK;
}

cslbm_status cslbm_batch_tune_results(const cslbm_batch* b, int max, int* shapes, float* ms, int* count)
{
    if (!b || !count || max < 0 || (max > 0 && (!shapes || !ms))) return bfail(CSLBM_EINVAL, "bad argument");
    const int n = (int)b->cand.size();
    *count = n;
    for (int i = 0; i < n && i < max; i++) {
        shapes[3 * i] = cslbm::batch::kTB[b->cand[i].tb];
        shapes[3 * i + 1] = b->cand[i].item;
        shapes[3 * i + 2] = b->cand[i].bps;
        ms[i] = b->cand_ms[i];
    }
    return CSLBM_OK;
}

cslbm_status cslbm_batch_check(cslbm_batch* b)
{
    if (!b) return bfail(CSLBM_EINVAL, "batch is null");
    int e = 0;
    BCUDA(cudaMemcpyAsync(&e, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    if (e) {
        BCUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
        BCUDA(cudaStreamSynchronize(b->stream));
        return bfail(CSLBM_ETIMEOUT, "the batch step's grid barrier ran out of time");
    }
    return CSLBM_OK;
}

cslbm_status cslbm_batch_launches(const cslbm_batch* b, long long* launches)
{
    if (!b || !launches) return bfail(CSLBM_EINVAL, "bad argument");
    *launches = b->launches;
    return CSLBM_OK;
}

cslbm_status cslbm_batch_destroy(cslbm_batch* b)
{
    if (!b) return bfail(CSLBM_EINVAL, "batch is null");
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaEventDestroy(b->ev_in);
    cudaEventDestroy(b->ev_out);
    cudaEventDestroy(b->t0);
    cudaEventDestroy(b->t1);
    cudaStreamDestroy(b->stream);
    for (cslbm_ctx* c : b->ctx) cslbm_destroy(c);
    delete b;
    return CSLBM_OK;
}

}  // extern "C"
