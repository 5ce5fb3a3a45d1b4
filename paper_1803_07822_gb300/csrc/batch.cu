// Batched form: many independent channels of uneven sizes advanced together,
// FP32 storage.
//
// Each channel is an ordinary context (its own workspace slice, metric,
// boundary velocities; every single-channel call works on it).  A time step
// of the whole batch is two launches over all channels: the momentum pass
// and the step pass of the gather form (k_momentum_flat / k_step_flat per
// node), whose blocks of TB consecutive nodes are laid end to end over the
// channels.  A block finds its channel by binary search in a table of
// per-channel first blocks held in shared memory; the channel's lattice,
// buffers and ping-pong parities come from a table in device memory.  The
// parity of the step inside a two-step cycle is a kernel argument, so two
// steps are captured once as a CUDA graph on the batch's own stream and
// replayed; the table is re-uploaded only when a channel's buffers moved
// (a metric update, a single-channel step).  TB is picked by
// cslbm_batch_tune, which times each candidate on the batch itself with the
// same step repeated from the same input (the state does not advance).
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

// first block of every channel (for block size TB) into shared memory, then
// the channel of this block
template <int TB>
__device__ __forceinline__ int load_blk0(const unsigned* __restrict__ starts, int nchan, unsigned* sb)
{
    for (int i = threadIdx.x; i < nchan; i += TB) sb[i] = starts[i];
    __syncthreads();
    return find_chan(sb, nchan, blockIdx.x);
}

template <int TB>
__global__ void __launch_bounds__(TB) k_batch_momentum(const Chan* __restrict__ tab, const unsigned* __restrict__ starts,
                                                        int nchan, int k)
{
    extern __shared__ unsigned sb_m[];
    const int c = load_blk0<TB>(starts, nchan, sb_m);
    const Chan& C = tab[c];
    const unsigned v = (blockIdx.x - sb_m[c]) * (unsigned)TB + threadIdx.x;
    if (v >= (unsigned)C.L.N) return;
    const unsigned n0 = C.L.n[0], n01 = n0 * C.L.n[1];
    const int z = (int)(v / n01), r = (int)(v - z * n01), y = r / (int)n0, x = r - y * (int)n0;
    momentum_node<float, float>(C.L, C.P[(C.pc0 + k) & 1], C.H[(C.hc0 + k) & 1], C.G, C.jf, x, y, z, v);
}

template <int TB>
__global__ void __launch_bounds__(TB) k_batch_step(const Chan* __restrict__ tab, const unsigned* __restrict__ starts,
                                                    int nchan, int k)
{
    extern __shared__ unsigned sb_s[];
    const int c = load_blk0<TB>(starts, nchan, sb_s);
    const Chan& C = tab[c];
    const unsigned v = (blockIdx.x - sb_s[c]) * (unsigned)TB + threadIdx.x;
    if (v >= (unsigned)C.L.N) return;
    const unsigned n0 = C.L.n[0], n01 = n0 * C.L.n[1];
    const int z = (int)(v / n01), r = (int)(v - z * n01), y = r / (int)n0, x = r - y * (int)n0;
    const int pi = (C.pc0 + k) & 1, hi = (C.hc0 + k) & 1;
    step_node<float, float>(C.L, C.P[pi], C.P[pi ^ 1], C.H[hi], C.H[hi ^ 1], C.G, C.jf, x, y, z, v);
}

constexpr int kTB[3] = {128, 256, 512};

}  // namespace batch
}  // namespace cslbm

using cslbm::batch::Chan;

struct cslbm_batch {
    int nb;
    std::vector<cslbm_ctx*> ctx;
    cudaStream_t user;    // the caller's stream
    cudaStream_t stream;  // the batch's own stream (graphs are captured on it)
    cudaEvent_t ev_in, ev_out, t0, t1;
    Chan* d_tab;          // [nb] in the workspace
    unsigned* d_starts;   // [3][nb]: first block of each channel for each block size
    std::vector<Chan> h_tab;
    std::vector<unsigned> h_starts;
    unsigned nblocks[3];
    int tb;                 // index into kTB
    cudaGraphExec_t graph;  // two steps
    int graph_tb;
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

void launch_step(cslbm_batch* b, int tb, int k, cudaStream_t s)
{
    using namespace cslbm::batch;
    const unsigned nbk = b->nblocks[tb];
    const unsigned* starts = b->d_starts + tb * b->nb;
    const size_t sm = b->nb * sizeof(unsigned);
    switch (tb) {
    case 0:
        k_batch_momentum<128><<<nbk, 128, sm, s>>>(b->d_tab, starts, b->nb, k);
        k_batch_step<128><<<nbk, 128, sm, s>>>(b->d_tab, starts, b->nb, k);
        break;
    case 1:
        k_batch_momentum<256><<<nbk, 256, sm, s>>>(b->d_tab, starts, b->nb, k);
        k_batch_step<256><<<nbk, 256, sm, s>>>(b->d_tab, starts, b->nb, k);
        break;
    default:
        k_batch_momentum<512><<<nbk, 512, sm, s>>>(b->d_tab, starts, b->nb, k);
        k_batch_step<512><<<nbk, 512, sm, s>>>(b->d_tab, starts, b->nb, k);
        break;
    }
}

cslbm_status make_graph(cslbm_batch* b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t g;
    BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    launch_step(b, b->tb, 0, b->stream);
    launch_step(b, b->tb, 1, b->stream);
    BCUDA(cudaStreamEndCapture(b->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(CSLBM_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
    b->graph_tb = b->tb;
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
    total += al(nb * sizeof(Chan)) + al(3 * nb * sizeof(unsigned));
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
    b->graph_tb = -1;
    b->tb = 1;
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
    b->d_starts = (unsigned*)(base + o);
    b->h_tab.resize(nb);
    b->h_starts.assign(3 * nb, 0);
    for (int t = 0; t < 3 && !st; t++) {
        unsigned acc = 0;
        for (int i = 0; i < nb; i++) {
            b->h_starts[t * nb + i] = acc;
            acc += (unsigned)((b->ctx[i]->N + cslbm::batch::kTB[t] - 1) / cslbm::batch::kTB[t]);
        }
        b->nblocks[t] = acc;
    }
    bool have_stream = false;
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
    if (!st && cudaMemcpyAsync(b->d_starts, b->h_starts.data(), 3 * nb * sizeof(unsigned), cudaMemcpyHostToDevice,
                               b->stream) != cudaSuccess)
        st = bfail(CSLBM_ECUDA, "table upload failed");
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
    if (!b->graph || b->graph_tb != b->tb)
        if (cslbm_status s = make_graph(b)) return s;
    for (int t = 0; t + 1 < nsteps; t += 2) {
        BCUDA(cudaGraphLaunch(b->graph, b->stream));
        b->launches += 4;
    }
    if (nsteps & 1) {
        launch_step(b, b->tb, 0, b->stream);
        BCUDA(cudaGetLastError());
        b->launches += 2;
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

cslbm_status cslbm_batch_tune(cslbm_batch* b, int reps, int* block_nodes, float* ms)
{
    if (!b || reps <= 0) return bfail(CSLBM_EINVAL, "bad argument");
    for (cslbm_ctx* c : b->ctx)
        if (!c->has_state) return bfail(CSLBM_ESTATE, "a channel of the batch has no state");
    BCUDA(cudaEventRecord(b->ev_in, b->user));
    BCUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    if (!table_current(b))
        if (cslbm_status s = upload_table(b)) return s;
    // the same step (parity 0) repeated: every repetition reads the current
    // state and writes the spare buffers, so the state does not advance
    float best = 1e30f;
    int best_t = b->tb;
    for (int t = 0; t < 3; t++) {
        launch_step(b, t, 0, b->stream);  // warm
        BCUDA(cudaEventRecord(b->t0, b->stream));
        for (int r = 0; r < reps; r++) launch_step(b, t, 0, b->stream);
        BCUDA(cudaEventRecord(b->t1, b->stream));
        BCUDA(cudaEventSynchronize(b->t1));
        BCUDA(cudaGetLastError());
        float e = 0.0f;
        BCUDA(cudaEventElapsedTime(&e, b->t0, b->t1));
        if (ms) ms[t] = e / reps;
        if (e < best) {
            best = e;
            best_t = t;
        }
    }
    b->tb = best_t;
    if (block_nodes) *block_nodes = cslbm::batch::kTB[best_t];
    BCUDA(cudaEventRecord(b->ev_out, b->stream));
    BCUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
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
