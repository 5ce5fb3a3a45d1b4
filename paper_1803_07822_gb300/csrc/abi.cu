// C ABI of the curved-space lattice Boltzmann library: context, workspace
// layout, host<->device staging and the order of kernel launches.  The
// kernels themselves live in kernels.cuh (one instantiation per format).
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>

#include "ctx.h"
#include "fp_convert.h"

namespace {

thread_local std::string g_err;

cslbm_status fail(cslbm_status s, const std::string& m)
{
    g_err = m;
    return s;
}

#define CUDA_TRY(call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail(CSLBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define LAUNCH_CHECK(what)                                                                          \
    do {                                                                                            \
        cudaError_t e_ = cudaGetLastError();                                                        \
        if (e_ != cudaSuccess) return fail(CSLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr long long kMaxChunk = 1LL << 20;  // nodes per host-transfer chunk
constexpr int kStagingDoubles = 24;           // per node: g6 + dg18

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t off_P[2], off_H[2], off_G[2], off_J, off_jf, off_face[6], off_scratch, off_done, off_staging, total;
    size_t s_bytes, r_bytes;
    long long N, chunk, face_n[6];
};

const cslbm_ops* ops_for(int storage)
{
    switch (storage) {
    case CSLBM_FP32: return &cslbm_ops_fp32;
    case CSLBM_FP16S: return &cslbm_ops_fp16;
    case CSLBM_BF16S: return &cslbm_ops_bf16;
    case CSLBM_FP64: return &cslbm_ops_fp64;
    default: return nullptr;
    }
}

cslbm_status validate(const cslbm_params* p)
{
    if (!p) return fail(CSLBM_EINVAL, "params is null");
    for (int a = 0; a < 3; a++) {
        if (p->n[a] < 1) return fail(CSLBM_EINVAL, "n must be >= 1 on every axis");
        for (int s = 0; s < 2; s++) {
            int b = s ? p->bc_hi[a] : p->bc_lo[a];
            if (b < CSLBM_PERIODIC || b > CSLBM_OUTFLOW) return fail(CSLBM_EINVAL, "unknown boundary rule");
        }
        if ((p->bc_lo[a] == CSLBM_PERIODIC) != (p->bc_hi[a] == CSLBM_PERIODIC))
            return fail(CSLBM_EINVAL, "an axis is periodic on both faces or on neither");
        if (p->bc_lo[a] != CSLBM_PERIODIC && p->n[a] < 3)
            return fail(CSLBM_EINVAL, "a non-periodic axis needs at least 3 nodes");
    }
    if (!(p->tau > 0.5)) return fail(CSLBM_EINVAL, "tau must exceed 1/2");
    if (!ops_for(p->storage)) return fail(CSLBM_EINVAL, "unknown storage format");
    if (p->step_kernel != CSLBM_STEP_AUTO && p->step_kernel != CSLBM_STEP_FLAT && p->step_kernel != CSLBM_STEP_ROWS)
        return fail(CSLBM_EINVAL, "unknown step kernel");
    if (p->n[2] > 65535) return fail(CSLBM_EINVAL, "n[2] must be at most 65535 (one launch row per plane)");
    // the step kernel indexes fields with 32-bit offsets (25 components of N)
    if (25LL * p->n[0] * p->n[1] * p->n[2] >= (1LL << 32))
        return fail(CSLBM_EINVAL, "lattice too large: at most 171,798,691 nodes per context");
    return CSLBM_OK;
}

Layout layout(const cslbm_params* p)
{
    Layout L{};
    L.N = (long long)p->n[0] * p->n[1] * p->n[2];
    L.s_bytes = p->storage == CSLBM_FP32 ? 4 : (p->storage == CSLBM_FP64 ? 8 : 2);
    L.r_bytes = p->storage == CSLBM_FP64 ? 8 : 4;
    L.chunk = L.N < kMaxChunk ? L.N : kMaxChunk;
    size_t o = 0;
    for (int k = 0; k < 2; k++) { L.off_P[k] = o; o += al(19 * L.N * L.s_bytes); }
    for (int k = 0; k < 2; k++) { L.off_H[k] = o; o += al(10 * L.N * L.r_bytes); }
    for (int k = 0; k < 2; k++) { L.off_G[k] = o; o += al(25 * L.N * L.r_bytes); }
    L.off_J = o; o += al(9 * L.N * L.r_bytes);
    L.off_jf = o; o += al(4 * L.N * L.r_bytes);
    for (int k = 0; k < 6; k++) {
        int a = k / 2;
        bool periodic = (k & 1 ? p->bc_hi[a] : p->bc_lo[a]) == CSLBM_PERIODIC;
        L.face_n[k] = (long long)p->n[(a + 1) % 3] * p->n[(a + 2) % 3];
        L.off_face[k] = o;
        if (!periodic) o += al(3 * L.face_n[k] * sizeof(double));
    }
    L.off_scratch = o; o += al(64 * sizeof(double));
    L.off_done = o; o += al((size_t)p->n[1] * p->n[2] * sizeof(unsigned));
    L.off_staging = o; o += al(kStagingDoubles * L.chunk * sizeof(double));
    L.total = o;
    return L;
}

__global__ void k_fill(double* p, long long n, double v)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
__global__ void k_fillf(float* p, long long n, float v)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

cslbm_status fill(cslbm_ctx* c, void* p, long long n, double v, bool fp64)
{
    unsigned nb = (unsigned)((n + 255) / 256);
    if (fp64) k_fill<<<nb, 256, 0, c->stream>>>((double*)p, n, v);
    else k_fillf<<<nb, 256, 0, c->stream>>>((float*)p, n, (float)v);
    LAUNCH_CHECK("fill");
    return CSLBM_OK;
}

// components k = 0..8 of cnt nodes from src [9][sstride] (FP64) into the stored
// Jacobian at nodes v0.., rounded to FP32 on the integer units unless the
// context computes in FP64 (the rounding of the chart-change kernels)
__global__ void k_store_jac(const double* __restrict__ src, long long sstride, void* __restrict__ J, long long N,
                            long long v0, long long cnt, int fp64)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    for (int k = 0; k < 9; k++) {
        const double x = src[k * sstride + t];
        if (fp64) ((double*)J)[k * N + v0 + t] = x;
        else ((float*)J)[k * N + v0 + t] = cslbm::f64_to_f32_rn(x);
    }
}

cslbm_status store_jacobian(cslbm_ctx* c, const double* src, long long sstride, long long v0, long long cnt)
{
    k_store_jac<<<(unsigned)((cnt + 255) / 256), 256, 0, c->stream>>>(src, sstride, c->J, c->N, v0, cnt,
                                                                      c->r_bytes == 8);
    LAUNCH_CHECK("Jacobian store");
    return CSLBM_OK;
}

// flat geometry into G[k]: sqrt g = 1, g^ij = delta, Gamma = 0
cslbm_status set_flat(cslbm_ctx* c, int k)
{
    const bool d = c->r_bytes == 8;
    char* g = (char*)c->G[k];
    CUDA_TRY(cudaMemsetAsync(g, 0, 25 * c->N * c->r_bytes, c->stream));
    const int ones[4] = {0, 1, 4, 6};  // sqrt g, g^00, g^11, g^22
    for (int i : ones) {
        cslbm_status s = fill(c, g + (size_t)i * c->N * c->r_bytes, c->N, 1.0, d);
        if (s) return s;
    }
    return CSLBM_OK;
}

// copy `ncomp` components of `cnt` nodes starting at v0 from a [ncomp][N]
// host or device array into the staging area as [ncomp][cnt].
cslbm_status stage_in(cslbm_ctx* c, const double* src, int ncomp, long long v0, long long cnt, double* dst)
{
    for (int k = 0; k < ncomp; k++)
        CUDA_TRY(cudaMemcpyAsync(dst + k * cnt, src + k * c->N + v0, cnt * sizeof(double), cudaMemcpyDefault,
                                 c->stream));
    return CSLBM_OK;
}

cslbm_status read_scratch(cslbm_ctx* c, double* out, int k)
{
    CUDA_TRY(cudaMemcpyAsync(out, c->scratch, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CSLBM_OK;
}

cslbm_status metric_flag(cslbm_ctx* c)
{
    int hbad = 0;
    CUDA_TRY(cudaMemcpyAsync(&hbad, c->scratch + 32, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->metric_check_pending = 0;
    if (hbad) return fail(CSLBM_EINVAL, "metric not positive definite (det g <= 0) at some node");
    return CSLBM_OK;
}

// Metric kernel over all nodes into G[dst].  The det g > 0 flag is read back
// at once (sync) or left pending for the next cslbm_check.
cslbm_status run_metric(cslbm_ctx* c, const double* g6, const double* dg18, int on_device, int dst, bool sync)
{
    int* bad = (int*)(c->scratch + 32);
    if (!c->metric_check_pending) CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    if (on_device) {
        c->ops->metric(c, g6, dg18, c->N, 0, c->N, dst, bad);
        c->launches++;
        LAUNCH_CHECK("metric kernel");
    } else {
        for (long long v0 = 0; v0 < c->N; v0 += c->chunk) {
            long long cnt = c->N - v0 < c->chunk ? c->N - v0 : c->chunk;
            cslbm_status s = stage_in(c, g6, 6, v0, cnt, c->staging);
            if (!s) s = stage_in(c, dg18, 18, v0, cnt, c->staging + 6 * cnt);
            if (s) return s;
            c->ops->metric(c, c->staging, c->staging + 6 * cnt, cnt, v0, cnt, dst, bad);
            c->launches++;
            LAUNCH_CHECK("metric kernel");
        }
    }
    if (sync) return metric_flag(c);
    c->metric_check_pending = 1;
    return CSLBM_OK;
}

}  // namespace

cslbm_status cslbm_record_error(cslbm_status s, const char* msg) { return fail(s, msg); }

namespace {

// The row-staged step pass: plan and tensor maps, when the storage, shape
// and device allow it (otherwise the flat pass serves).
void rows_prepare(cslbm_ctx* c)
{
    cslbm_rows& R = c->rows;
    R.ok = 0;
    R.fused_ok = 0;
    R.epoch = 0;
    R.test_wait_ns = 0;
    R.test_withhold = -1;
    if (c->p.step_kernel == CSLBM_STEP_FLAT || c->p.storage == CSLBM_FP64) return;
    int max_smem = 0;
    if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess) return;
    if (!cslbm::rows::make_plan(c->n, c->p.bc_lo[1] == CSLBM_PERIODIC, c->p.bc_lo[2] == CSLBM_PERIODIC,
                                (int)c->s_bytes, max_smem, R.plan))
        return;
    typedef CUresult (*encode_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess || !fn ||
        q != cudaDriverEntryPointSuccess)
        return;
    encode_fn encode = (encode_fn)fn;
    const cuuint64_t n0 = c->n[0], n1 = c->n[1], n2 = c->n[2], N = c->N, sb = c->s_bytes;
    const cuuint32_t TR = R.plan.TR, NT = cslbm::rows::NT;
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    auto mk = [&](CUtensorMap* m, CUtensorMapDataType t, cuuint32_t rank, void* base, const cuuint64_t* dims,
                  const cuuint64_t* strides, const cuuint32_t* box) {
        return encode(m, t, rank, base, dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    const CUtensorMapDataType tpop = sb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    bool ok = true;
    for (int k = 0; k < 2 && ok; k++) {
        const cuuint64_t pd[4] = {n0, n1, n2, 19}, ps[3] = {n0 * sb, n0 * n1 * sb, N * sb};
        const cuuint32_t pb[4] = {(cuuint32_t)n0, TR, 1, 1}, pb3[4] = {(cuuint32_t)n0, TR, 1, 3};
        ok = ok && mk(&R.pop[k], tpop, 4, c->P[k], pd, ps, pb);
        ok = ok && mk(&R.pop3[k], tpop, 4, c->P[k], pd, ps, pb3);
        const cuuint64_t gd[2] = {N, 25}, gs[1] = {N * 4};
        const cuuint32_t gb[2] = {NT, 25};
        ok = ok && mk(&R.geo[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->G[k], gd, gs, gb);
        const cuuint64_t hd[2] = {N, 10};
        const cuuint32_t hb[2] = {NT, 10};
        ok = ok && mk(&R.hist[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->H[k], hd, gs, hb);
        const cuuint32_t g1b[2] = {NT, 1}, h4b[2] = {NT, 4};
        ok = ok && mk(&R.geo1[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->G[k], gd, gs, g1b);
        ok = ok && mk(&R.hist4[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->H[k], hd, gs, h4b);
    }
    // rho u viewed as lines of JL floats, so that the TR + 2 contiguous rows of
    // a layer are JR lines of up to 1 KB (a view with one 16-byte node per
    // line would make the copy engine move hundreds of 16-byte lines)
    const cuuint64_t JL = R.plan.JL;
    const cuuint64_t jd[2] = {JL, 4 * N / JL}, js[1] = {JL * 4};
    const cuuint32_t jb[2] = {(cuuint32_t)JL, (cuuint32_t)R.plan.JR};
    ok = ok && mk(&R.jf, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->jf, jd, js, jb);
    // the same lines per plane, three planes per box
    const cuuint64_t jd3[3] = {JL, 4 * n0 * n1 / JL, n2}, js3[2] = {JL * 4, n0 * n1 * 16};
    const cuuint32_t jb3[3] = {(cuuint32_t)JL, (cuuint32_t)R.plan.JR, 3};
    ok = ok && mk(&R.jf3, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->jf, jd3, js3, jb3);
    if (!ok) return;
    R.ok = 1;
    // the fused form: momentum and step in one cooperative launch
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
    if (c->p.step_kernel == CSLBM_STEP_AUTO && coop && c->p.bc_lo[2] != CSLBM_PERIODIC &&
        cslbm::rows::fused_layout(R.plan, (int)c->s_bytes, max_smem, R.off_m, R.off_sg, R.off_h4, R.off_js,
                                  R.fused_bytes))
        R.fused_ok = 1;
}

}  // namespace

extern "C" {

cslbm_status cslbm_workspace_bytes(const cslbm_params* p, size_t* bytes)
{
    if (cslbm_status s = validate(p)) return s;
    if (!bytes) return fail(CSLBM_EINVAL, "bytes is null");
    *bytes = layout(p).total;
    return CSLBM_OK;
}

cslbm_status cslbm_create(const cslbm_params* p, void* ws, size_t bytes, void* stream, cslbm_ctx** out)
{
    if (cslbm_status s = validate(p)) return s;
    if (!ws || !out) return fail(CSLBM_EINVAL, "workspace or out is null");
    if ((uintptr_t)ws & 255) return fail(CSLBM_EINVAL, "workspace must be 256-byte aligned");
    Layout L = layout(p);
    if (bytes < L.total) return fail(CSLBM_ENOMEM, "workspace smaller than cslbm_workspace_bytes");
    cslbm_ctx* c = new cslbm_ctx();
    c->p = *p;
    for (int a = 0; a < 3; a++) c->n[a] = p->n[a];
    c->N = L.N;
    c->theta = p->theta > 0 ? p->theta : 1.0 / 3.0;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    c->s_bytes = L.s_bytes;
    c->r_bytes = L.r_bytes;
    char* b = (char*)ws;
    for (int k = 0; k < 2; k++) {
        c->P[k] = b + L.off_P[k];
        c->H[k] = b + L.off_H[k];
        c->G[k] = b + L.off_G[k];
    }
    c->J = b + L.off_J;
    c->jf = b + L.off_jf;
    for (int k = 0; k < 6; k++) {
        int a = k / 2;
        bool periodic = (k & 1 ? p->bc_hi[a] : p->bc_lo[a]) == CSLBM_PERIODIC;
        c->face[k] = periodic ? nullptr : (double*)(b + L.off_face[k]);
        c->face_n[k] = L.face_n[k];
    }
    c->scratch = (double*)(b + L.off_scratch);
    c->rows.done = (unsigned*)(b + L.off_done);
    c->staging = (double*)(b + L.off_staging);
    c->chunk = L.chunk;
    c->pc = c->hc = c->gc = 0;
    c->has_state = 0;
    c->ops = ops_for(p->storage);
    cslbm_status s = CSLBM_OK;
    if (cudaMemsetAsync(ws, 0, L.total, c->stream) != cudaSuccess) s = fail(CSLBM_ECUDA, "workspace memset failed");
    if (!s) s = set_flat(c, 0);
    if (!s) s = set_flat(c, 1);
    if (!s) {
        for (int i : {0, 4, 8}) {
            s = fill(c, (char*)c->J + (size_t)i * c->N * c->r_bytes, c->N, 1.0, c->r_bytes == 8);
            if (s) break;
        }
    }
    if (s) {
        delete c;
        return s;
    }
    rows_prepare(c);
    cudaGetLastError();  // a pass that could not be prepared leaves no error behind
    *out = c;
    return CSLBM_OK;
}

cslbm_status cslbm_destroy(cslbm_ctx* c)
{
    if (!c) return fail(CSLBM_EINVAL, "ctx is null");
    cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    delete c;
    return CSLBM_OK;
}

cslbm_status cslbm_set_metric(cslbm_ctx* c, const double* g6, const double* dg18, int on_device)
{
    if (!c || !g6 || !dg18) return fail(CSLBM_EINVAL, "null argument");
    return run_metric(c, g6, dg18, on_device, c->gc, true);
}

static bool is_device_memory(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cslbm_status cslbm_transform_interp_scratch_bytes(const cslbm_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return fail(CSLBM_EINVAL, "null argument");
    *bytes = 20 * (size_t)c->N * c->r_bytes;
    return CSLBM_OK;
}

cslbm_status cslbm_update_metric_interp(cslbm_ctx* c, const double* g6, const double* dg18, const double* Jnew9,
                                        const double* psi3, void* scratch, size_t scratch_bytes)
{
    if (!c || !g6 || !dg18 || !Jnew9 || !psi3) return fail(CSLBM_EINVAL, "null argument");
    if (!c->has_state) return fail(CSLBM_ESTATE, "update_metric_interp before init_equilibrium");
    if (!scratch || scratch_bytes < 20 * (size_t)c->N * c->r_bytes) return fail(CSLBM_ENOMEM, "scratch too small");
    for (const void* q : {(const void*)g6, (const void*)dg18, (const void*)Jnew9, (const void*)psi3, (const void*)scratch})
        if (!is_device_memory(q)) return fail(CSLBM_EINVAL, "every array of update_metric_interp is device memory");
    if (cslbm_status s = run_metric(c, g6, dg18, 1, 1 - c->gc, false)) return s;
    c->ops->transform_interp(c, Jnew9, psi3, scratch);
    c->launches += 2;
    LAUNCH_CHECK("interpolating transform kernels");
    if (cslbm_status s = store_jacobian(c, Jnew9, c->N, 0, c->N)) return s;
    c->pc ^= 1;
    c->hc ^= 1;
    c->gc ^= 1;
    return CSLBM_OK;
}

cslbm_status cslbm_set_jacobian(cslbm_ctx* c, const double* J9, int on_device)
{
    if (!c || !J9) return fail(CSLBM_EINVAL, "null argument");
    if (on_device) return store_jacobian(c, J9, c->N, 0, c->N);
    for (long long v0 = 0; v0 < c->N; v0 += c->chunk) {
        const long long cnt = c->N - v0 < c->chunk ? c->N - v0 : c->chunk;
        if (cslbm_status s = stage_in(c, J9, 9, v0, cnt, c->staging)) return s;
        if (cslbm_status s = store_jacobian(c, c->staging, cnt, v0, cnt)) return s;
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CSLBM_OK;
}

cslbm_status cslbm_update_metric(cslbm_ctx* c, const double* g6, const double* dg18, const double* Jnew9,
                                 int on_device)
{
    if (!c || !g6 || !dg18 || !Jnew9) return fail(CSLBM_EINVAL, "null argument");
    if (!c->has_state) return fail(CSLBM_ESTATE, "update_metric before init_equilibrium");
    if (on_device) {
        // metric and transformation in one pass
        int* bad = (int*)(c->scratch + 32);
        if (!c->metric_check_pending) CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
        c->ops->chart_change(c, g6, dg18, Jnew9, bad);
        c->launches++;
        LAUNCH_CHECK("chart-change kernel");
        c->metric_check_pending = 1;
    } else {
        if (cslbm_status s = run_metric(c, g6, dg18, on_device, 1 - c->gc, false)) return s;
        for (long long v0 = 0; v0 < c->N; v0 += c->chunk) {
            long long cnt = c->N - v0 < c->chunk ? c->N - v0 : c->chunk;
            if (cslbm_status s = stage_in(c, Jnew9, 9, v0, cnt, c->staging)) return s;
            c->ops->transform(c, c->staging, cnt, v0, cnt);
            c->launches++;
            LAUNCH_CHECK("transform kernel");
        }
    }
    c->pc ^= 1;
    c->hc ^= 1;
    c->gc ^= 1;
    return CSLBM_OK;
}

cslbm_status cslbm_update_metric_mixed(cslbm_ctx* c, const double* g6, const float* dg18, const float* Jnew9)
{
    if (!c || !g6 || !dg18 || !Jnew9) return fail(CSLBM_EINVAL, "null argument");
    if (c->r_bytes == 8) return fail(CSLBM_EINVAL, "FP64 storage takes its derivatives and Jacobian in FP64");
    for (const void* q : {(const void*)g6, (const void*)dg18, (const void*)Jnew9})
        if (!is_device_memory(q)) return fail(CSLBM_EINVAL, "every array of update_metric_mixed is device memory");
    if (!c->has_state) return fail(CSLBM_ESTATE, "update_metric before init_equilibrium");
    int* bad = (int*)(c->scratch + 32);
    if (!c->metric_check_pending) CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    c->ops->chart_change_mixed(c, g6, dg18, Jnew9, bad);
    c->launches++;
    LAUNCH_CHECK("chart-change kernel");
    c->metric_check_pending = 1;
    c->pc ^= 1;
    c->hc ^= 1;
    c->gc ^= 1;
    return CSLBM_OK;
}

cslbm_status cslbm_init_equilibrium(cslbm_ctx* c, const double* rho, const double* u3, int on_device)
{
    if (!c) return fail(CSLBM_EINVAL, "ctx is null");
    for (int k = 0; k < 2; k++) {
        CUDA_TRY(cudaMemsetAsync(c->P[k], 0, 19 * c->N * c->s_bytes, c->stream));
        CUDA_TRY(cudaMemsetAsync(c->H[k], 0, 10 * c->N * c->r_bytes, c->stream));
    }
    if (on_device || (!rho && !u3)) {
        c->ops->init_scatter(c, rho, u3, c->N, 0, c->N);
        LAUNCH_CHECK("init kernel");
    } else {
        for (long long v0 = 0; v0 < c->N; v0 += c->chunk) {
            long long cnt = c->N - v0 < c->chunk ? c->N - v0 : c->chunk;
            double* r = rho ? c->staging : nullptr;
            double* u = u3 ? c->staging + cnt : nullptr;
            if (rho)
                if (cslbm_status s = stage_in(c, rho, 1, v0, cnt, r)) return s;
            if (u3)
                if (cslbm_status s = stage_in(c, u3, 3, v0, cnt, u)) return s;
            c->ops->init_scatter(c, r, u, cnt, v0, cnt);
            LAUNCH_CHECK("init kernel");
        }
    }
    // forcing of the initial state, F(x, -dt) := F(x, 0)
    c->ops->momentum_field(c);
    LAUNCH_CHECK("momentum kernel");
    c->ops->step(c, 1);
    LAUNCH_CHECK("forcing kernel");
    c->hc ^= 1;
    c->ops->half_shift(c);
    c->launches += 3;
    LAUNCH_CHECK("shift kernel");
    c->has_state = 1;
    if (!on_device && (rho || u3)) CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CSLBM_OK;
}

cslbm_status cslbm_set_boundary_velocity(cslbm_ctx* c, int axis, int side, const double* u3, int on_device)
{
    if (!c || axis < 0 || axis > 2 || side < 0 || side > 1) return fail(CSLBM_EINVAL, "bad face");
    int k = axis * 2 + side;
    int bc = side ? c->p.bc_hi[axis] : c->p.bc_lo[axis];
    if (bc != CSLBM_WALL && bc != CSLBM_INFLOW) return fail(CSLBM_EINVAL, "face is not a wall or inflow face");
    size_t bytes = 3 * c->face_n[k] * sizeof(double);
    if (!u3) CUDA_TRY(cudaMemsetAsync(c->face[k], 0, bytes, c->stream));
    else CUDA_TRY(cudaMemcpyAsync(c->face[k], u3, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream));
    if (u3 && !on_device) CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CSLBM_OK;
}

cslbm_status cslbm_step(cslbm_ctx* c, int nsteps)
{
    if (!c || nsteps < 0) return fail(CSLBM_EINVAL, "bad argument");
    if (!c->has_state) return fail(CSLBM_ESTATE, "step before init_equilibrium");
    for (int t = 0; t < nsteps; t++) {
        if (c->prof) {
            cudaEvent_t e[2];
            CUDA_TRY(cudaEventCreate(&e[0]));
            CUDA_TRY(cudaEventCreate(&e[1]));
            c->ev.push_back(e[0]);
            c->ev.push_back(e[1]);
            CUDA_TRY(cudaEventRecord(e[0], c->stream));
        }
        c->launches += c->ops->step(c, 0);
        LAUNCH_CHECK("step kernel");
        if (c->prof) {
            CUDA_TRY(cudaEventRecord(c->ev.back(), c->stream));
            c->prof_steps++;
        }
        c->pc ^= 1;
        c->hc ^= 1;
    }
    return CSLBM_OK;
}

cslbm_status cslbm_get_moments(cslbm_ctx* c, double* rho, double* u3, int cartesian, int on_device)
{
    if (!c || (!rho && !u3)) return fail(CSLBM_EINVAL, "null argument");
    if (!c->has_state) return fail(CSLBM_ESTATE, "no state");
    if (on_device) {
        c->ops->readout(c, rho, u3, c->N, 0, c->N, cartesian);
        c->launches++;
        LAUNCH_CHECK("readout kernel");
        return CSLBM_OK;
    }
    for (long long v0 = 0; v0 < c->N; v0 += c->chunk) {
        long long cnt = c->N - v0 < c->chunk ? c->N - v0 : c->chunk;
        double* r = c->staging;
        double* u = c->staging + cnt;
        c->ops->readout(c, rho ? r : nullptr, u3 ? u : nullptr, cnt, v0, cnt, cartesian);
        c->launches++;
        LAUNCH_CHECK("readout kernel");
        if (rho) CUDA_TRY(cudaMemcpyAsync(rho + v0, r, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (u3)
            for (int a = 0; a < 3; a++)
                CUDA_TRY(cudaMemcpyAsync(u3 + a * c->N + v0, u + a * cnt, cnt * sizeof(double), cudaMemcpyDeviceToHost,
                                         c->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CSLBM_OK;
}

cslbm_status cslbm_total_mass(cslbm_ctx* c, double* out)
{
    if (!c || !out) return fail(CSLBM_EINVAL, "null argument");
    if (!c->has_state) return fail(CSLBM_ESTATE, "no state");
    CUDA_TRY(cudaMemsetAsync(c->scratch, 0, 8 * sizeof(double), c->stream));
    c->ops->mass(c, c->scratch);
    c->launches++;
    LAUNCH_CHECK("mass kernel");
    return read_scratch(c, out, 1);
}

cslbm_status cslbm_wall_force(cslbm_ctx* c, int axis, int side, double out3[3])
{
    if (!c || !out3 || axis < 0 || axis > 2 || side < 0 || side > 1) return fail(CSLBM_EINVAL, "bad argument");
    if (!c->has_state) return fail(CSLBM_ESTATE, "no state");
    CUDA_TRY(cudaMemsetAsync(c->scratch, 0, 8 * sizeof(double), c->stream));
    c->ops->wall_force(c, axis, side, c->scratch);
    c->launches++;
    LAUNCH_CHECK("wall-force kernel");
    return read_scratch(c, out3, 3);
}

cslbm_status cslbm_check(cslbm_ctx* c)
{
    if (!c) return fail(CSLBM_EINVAL, "ctx is null");
    if (!c->has_state) return fail(CSLBM_ESTATE, "no state");
    if (c->metric_check_pending)
        if (cslbm_status s = metric_flag(c)) return s;
    {
        int terr = 0;
        CUDA_TRY(cudaMemcpyAsync(&terr, step_error_flag(c), sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (terr) {
            CUDA_TRY(cudaMemsetAsync(step_error_flag(c), 0, sizeof(int), c->stream));
            // the fused pass's publication counts are no longer in step with
            // its launch count: start both again
            if (c->rows.ok) {
                CUDA_TRY(cudaMemsetAsync(c->rows.done, 0, (size_t)c->n[1] * c->n[2] * sizeof(unsigned), c->stream));
                c->rows.epoch = 0;
            }
            char m[96];
            snprintf(m, sizeof m, "a bounded wait of the row-staged step pass ran out (code %d)", terr);
            return fail(CSLBM_ETIMEOUT, m);
        }
    }
    CUDA_TRY(cudaMemsetAsync(c->scratch, 0, 8 * sizeof(double), c->stream));
    c->ops->check(c, c->scratch);
    c->launches++;
    LAUNCH_CHECK("check kernel");
    double bad = 0.0;
    if (cslbm_status s = read_scratch(c, &bad, 1)) return s;
    if (bad > 0.0) {
        char m[96];
        snprintf(m, sizeof m, "%.0f nodes with non-finite density or |v| > 0.3", bad);
        return fail(CSLBM_EUNSTABLE, m);
    }
    return CSLBM_OK;
}

cslbm_status cslbm_test_withhold_publication(cslbm_ctx* c, int iteration, long long wait_ns)
{
    if (!c) return fail(CSLBM_EINVAL, "ctx is null");
    if (!c->rows.fused_ok || c->p.step_kernel != CSLBM_STEP_AUTO)
        return fail(CSLBM_EINVAL, "the fused step pass does not apply to this lattice");
    if (iteration < 0 || wait_ns <= 0 || wait_ns > (long long)cslbm::rows::kWaitNs)
        return fail(CSLBM_EINVAL, "iteration must be >= 0 and wait_ns in (0, 5e8]");
    c->rows.test_withhold = iteration;
    c->rows.test_wait_ns = (unsigned long long)wait_ns;
    return CSLBM_OK;
}

cslbm_status cslbm_state_bytes(const cslbm_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return fail(CSLBM_EINVAL, "null argument");
    *bytes = 19 * c->N * c->s_bytes + 10 * c->N * c->r_bytes;
    return CSLBM_OK;
}

cslbm_status cslbm_save_state(cslbm_ctx* c, void* buf, size_t bytes, int on_device)
{
    size_t need = 0;
    if (cslbm_status s = cslbm_state_bytes(c, &need)) return s;
    if (!buf || bytes < need) return fail(CSLBM_EINVAL, "buffer too small");
    if (!c->has_state) return fail(CSLBM_ESTATE, "no state");
    size_t pb = 19 * c->N * c->s_bytes;
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CUDA_TRY(cudaMemcpyAsync(buf, c->P[c->pc], pb, k, c->stream));
    CUDA_TRY(cudaMemcpyAsync((char*)buf + pb, c->H[c->hc], need - pb, k, c->stream));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CSLBM_OK;
}

cslbm_status cslbm_load_state(cslbm_ctx* c, const void* buf, size_t bytes, int on_device)
{
    size_t need = 0;
    if (cslbm_status s = cslbm_state_bytes(c, &need)) return s;
    if (!buf || bytes < need) return fail(CSLBM_EINVAL, "buffer too small");
    size_t pb = 19 * c->N * c->s_bytes;
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CUDA_TRY(cudaMemcpyAsync(c->P[c->pc], buf, pb, k, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->H[c->hc], (const char*)buf + pb, need - pb, k, c->stream));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->has_state = 1;
    return CSLBM_OK;
}

cslbm_status cslbm_profile_enable(cslbm_ctx* c, int enable)
{
    if (!c) return fail(CSLBM_EINVAL, "ctx is null");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    c->prof = enable ? 1 : 0;
    c->prof_steps = 0;
    c->launches = 0;
    return CSLBM_OK;
}

cslbm_status cslbm_profile_read(cslbm_ctx* c, double* step_ms, long long* nsteps, long long* launches)
{
    if (!c) return fail(CSLBM_EINVAL, "ctx is null");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    double total = 0.0;
    for (size_t k = 0; k + 1 < c->ev.size(); k += 2) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
        total += ms;
    }
    if (step_ms) *step_ms = total;
    if (nsteps) *nsteps = c->prof_steps;
    if (launches) *launches = c->launches;
    return CSLBM_OK;
}

const char* cslbm_last_error(void) { return g_err.c_str(); }

}  // extern "C"
