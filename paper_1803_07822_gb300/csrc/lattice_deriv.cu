// Isotropic lattice derivatives of FP64 fields (App. D) on the device, and
// the geometry of a context from its metric alone.
//
// With the D3Q19 weights w_l and velocities c_l (lattice units):
//   G_i f(x) = (1/c_s^2) sum_l w_l c_l^i f(x + c_l)            second order
//   L f(x)   = (2/c_s^2) sum_l w_l (f(x + c_l) - f(x))         second order
//   d_i f(x) = G_i[f - (c_s^2/2) L f](x)                        fourth order
// (the third-order term of G_i is (c_s^2/2) d_i Lap f: the fourth moment of
// the D3Q19 weights is isotropic).  Beyond a non-periodic face the field is
// continued by the polynomial of degree `order` through the order + 1 nodes
// nearest the face, axis by axis (tensor product at edges and corners).
//
// Two kernels: k_pad writes F = f - (c_s^2/2) L f (order 4) or the continued f
// (order 2) on the lattice padded by one site along every axis with a
// non-periodic face, k_grad forms G_i F at every node from the nine opposite
// pairs.  One thread per (padded site or node, component); FP64 throughout.
#include <cstdint>
#include <string>

#include "ctx.h"
#include "lbm_device.cuh"

cslbm_status cslbm_record_error(cslbm_status s, const char* msg);

namespace cslbm {
namespace lder {

constexpr int TBL = 256;
constexpr double kCs2 = 1.0 / 3.0;

struct Box {
    int n[3];
    int plo[3], phi[3];  // low / high face periodic
    int pad[3];          // 1 on an axis with a non-periodic face
    int ne[3];           // padded extents n + 2 pad
    long long N, Ne;
};

// Weight of node k (k = 0 the face node, counting inward) in the value t = 1
// or 2 sites beyond the face: the polynomial of degree `order` through the
// nodes 0..order, evaluated at -t (Lagrange form, worked out).
__device__ __forceinline__ double cont_weight(int order, int t, int k)
{
    if (order == 2) {
        const double a[3] = {3.0, -3.0, 1.0}, b[3] = {6.0, -8.0, 3.0};
        return t == 1 ? a[k] : b[k];
    }
    const double a[5] = {5.0, -10.0, 10.0, -5.0, 1.0}, b[5] = {15.0, -40.0, 45.0, -24.0, 5.0};
    return t == 1 ? a[k] : b[k];
}

__device__ __forceinline__ bool wrap(const Box& B, int a, int& r)
{
    if (r < 0 && B.plo[a]) r += B.n[a];
    else if (r >= B.n[a] && B.phi[a]) r -= B.n[a];
    return r >= 0 && r < B.n[a];
}

// the continued field at a site up to two steps beyond a face: the terms of
// every out-of-range axis multiplied out
__device__ __noinline__ double site_far(const Box& B, const double* __restrict__ f, int order, int x, int y, int z)
{
    int c[3][5], m[3];
    double w[3][5];
    const int r[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int ra = r[a];
        if (wrap(B, a, ra)) {
            m[a] = 1;
            c[a][0] = ra;
            w[a][0] = 1.0;
            continue;
        }
        const bool lo = ra < 0;
        const int t = lo ? -ra : ra - (B.n[a] - 1);
        m[a] = order + 1;
        for (int k = 0; k <= order; k++) {
            c[a][k] = lo ? k : B.n[a] - 1 - k;
            w[a][k] = cont_weight(order, t, k);
        }
    }
    double v = 0.0;
    for (int k = 0; k < m[2]; k++)
        for (int j = 0; j < m[1]; j++) {
            double row = 0.0;
            const long long base = ((long long)c[2][k] * B.n[1] + c[1][j]) * B.n[0];
            for (int i = 0; i < m[0]; i++) row += w[0][i] * f[base + c[0][i]];
            v += w[2][k] * w[1][j] * row;
        }
    return v;
}

__device__ __forceinline__ double site(const Box& B, const double* __restrict__ f, int order, int x, int y, int z)
{
    int xs = x, ys = y, zs = z;
    if (wrap(B, 0, xs) && wrap(B, 1, ys) && wrap(B, 2, zs))
        return __ldg(f + ((long long)zs * B.n[1] + ys) * B.n[0] + xs);
    return site_far(B, f, order, x, y, z);
}

// a site whose whole stencil resolves without continuation (periodic wrap only)
__device__ __forceinline__ bool inner(const Box& B, int a, int r)
{
    return r >= 0 && r < B.n[a] && (r >= 1 || B.plo[a]) && (r <= B.n[a] - 2 || B.phi[a]);
}
__device__ __forceinline__ long long nb_index(const Box& B, int x, int y, int z)
{
    wrap(B, 0, x);
    wrap(B, 1, y);
    wrap(B, 2, z);
    return ((long long)z * B.n[1] + y) * B.n[0] + x;
}

// F = f - (c_s^2/2) L f = f0 - sum_l w_l (f_l - f0) (order 4), or the
// continued f (order 2), at every site of the padded lattice; component
// blockIdx.y
__global__ void __launch_bounds__(TBL) k_pad(const __grid_constant__ Box B, const double* __restrict__ f, int order,
                                             double* __restrict__ F)
{
    // 32-bit site arithmetic (the padded lattice has fewer than 2^32 sites)
    const unsigned s = blockIdx.x * TBL + threadIdx.x;
    if (s >= (unsigned)B.Ne) return;
    const double* fc = f + (long long)blockIdx.y * B.N;
    const unsigned ne0 = B.ne[0], ne1 = B.ne[1], row = s / ne0, zr = row / ne1;
    const int x = (int)(s - row * ne0) - B.pad[0];
    const int y = (int)(row - zr * ne1) - B.pad[1];
    const int z = (int)zr - B.pad[2];
    // with sum_{l>0} w_l = 2/3, w = 1/18 on the six faces, 1/36 on the twelve
    // edges: F = (5/3) f0 - (S_faces + S_edges / 2) / 18
    double f0, sf = 0.0, se = 0.0;
    if (inner(B, 0, x) && inner(B, 1, y) && inner(B, 2, z)) {
        // neighbour offsets per axis, wrapped on periodic axes (as nb_index)
        const unsigned n0 = B.n[0], n01 = n0 * (unsigned)B.n[1];
        unsigned o[3][3];
        const int r[3] = {x, y, z};
        const unsigned st[3] = {1u, n0, n01};
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int c = -1; c <= 1; c++) {
                int q = r[a] + c;
                wrap(B, a, q);
                o[a][c + 1] = (unsigned)q * st[a];
            }
        f0 = __ldg(fc + (o[2][1] + o[1][1] + o[0][1]));
        if (order == 4) {
#pragma unroll
            for (int l = 1; l < Q; l++) {
                const double fl = __ldg(fc + (o[2][cvec(l, 2) + 1] + o[1][cvec(l, 1) + 1] + o[0][cvec(l, 0) + 1]));
                if (l <= 6) sf += fl;
                else se += fl;
            }
        }
    } else {
        f0 = site(B, fc, order, x, y, z);
        if (order == 4) {
#pragma unroll
            for (int l = 1; l < Q; l++) {
                const double fl = site(B, fc, order, x + cvec(l, 0), y + cvec(l, 1), z + cvec(l, 2));
                if (l <= 6) sf += fl;
                else se += fl;
            }
        }
    }
    const double out = order == 4 ? fma(5.0 / 3.0, f0, -fma(0.5, se, sf) * (1.0 / 18.0)) : f0;
    F[(long long)blockIdx.y * B.Ne + s] = out;
}

// a site at most one step beyond a face, in the padded lattice
__device__ __forceinline__ long long pad_index(const Box& B, int x, int y, int z)
{
    wrap(B, 0, x);
    wrap(B, 1, y);
    wrap(B, 2, z);
    return ((long long)(z + B.pad[2]) * B.ne[1] + (y + B.pad[1])) * B.ne[0] + (x + B.pad[0]);
}

// d_k f_c = G_k F at every node, over the nine opposite pairs:
// out[(k ncomp + c) N + v]
__global__ void __launch_bounds__(TBL) k_grad(const __grid_constant__ Box B, int ncomp, const double* __restrict__ F,
                                              double* __restrict__ out)
{
    const unsigned v = blockIdx.x * TBL + threadIdx.x;
    if (v >= (unsigned)B.N) return;
    const int c = blockIdx.y;
    const double* Fc = F + (long long)c * B.Ne;
    const unsigned n0 = B.n[0], n1 = B.n[1], row = v / n0, zr = row / n1;
    const int x = (int)(v - row * n0), y = (int)(row - zr * n1), z = (int)zr;
    // offsets of the sites r + c per axis in the padded lattice (as pad_index)
    unsigned o[3][3];
    {
        const int r[3] = {x, y, z};
        const unsigned st[3] = {1u, (unsigned)B.ne[0], (unsigned)B.ne[0] * (unsigned)B.ne[1]};
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int cc = -1; cc <= 1; cc++) {
                int q = r[a] + cc;
                wrap(B, a, q);
                o[a][cc + 1] = (unsigned)(q + B.pad[a]) * st[a];
            }
    }
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const int l = 2 * k + 1, cx = cvec(l, 0), cy = cvec(l, 1), cz = cvec(l, 2);
        const double d = __ldg(Fc + (o[2][cz + 1] + o[1][cy + 1] + o[0][cx + 1])) -
                         __ldg(Fc + (o[2][1 - cz] + o[1][1 - cy] + o[0][1 - cx]));
        const double wd = wq(l) / kCs2;
        if (cx) g0 = fma(cx * wd, d, g0);
        if (cy) g1 = fma(cy * wd, d, g1);
        if (cz) g2 = fma(cz * wd, d, g2);
    }
    out[((long long)0 * ncomp + c) * B.N + v] = g0;
    out[((long long)1 * ncomp + c) * B.N + v] = g1;
    out[((long long)2 * ncomp + c) * B.N + v] = g2;
}

Box box_of(const cslbm_ctx* c, int order)
{
    Box B;
    B.N = c->N;
    B.Ne = 1;
    for (int a = 0; a < 3; a++) {
        B.n[a] = c->n[a];
        B.plo[a] = c->p.bc_lo[a] == CSLBM_PERIODIC;
        B.phi[a] = c->p.bc_hi[a] == CSLBM_PERIODIC;
        B.pad[a] = (B.plo[a] && B.phi[a]) ? 0 : 1;
        B.ne[a] = B.n[a] + 2 * B.pad[a];
        B.Ne *= B.ne[a];
    }
    return B;
}

cslbm_status lfail(cslbm_status s, const std::string& m) { return cslbm_record_error(s, m.c_str()); }

cslbm_status check_order(const cslbm_ctx* c, int order)
{
    if (order != 2 && order != 4) return lfail(CSLBM_EINVAL, "order must be 2 or 4");
    for (int a = 0; a < 3; a++)
        if (c->n[a] < 2) return lfail(CSLBM_EINVAL, "every axis needs at least 2 nodes");
    for (int a = 0; a < 3; a++)
        if ((c->p.bc_lo[a] != CSLBM_PERIODIC || c->p.bc_hi[a] != CSLBM_PERIODIC) && c->n[a] < order + 1)
            return lfail(CSLBM_EINVAL, "an axis with a non-periodic face needs at least order + 1 nodes");
    return CSLBM_OK;
}

bool device_memory(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t pad_bytes(const cslbm_ctx* c, int ncomp, int order)
{
    return (size_t)ncomp * (size_t)box_of(c, order).Ne * sizeof(double);
}

cslbm_status gradient(cslbm_ctx* c, const double* f, int ncomp, int order, double* out, void* scratch, size_t bytes)
{
    if (!c || !f || !out || ncomp < 1 || ncomp > 65535) return lfail(CSLBM_EINVAL, "bad argument");
    if (cslbm_status s = check_order(c, order)) return s;
    const size_t need = pad_bytes(c, ncomp, order);
    if (!scratch || bytes < need) return lfail(CSLBM_ENOMEM, "scratch smaller than required");
    if (!device_memory(f) || !device_memory(out) || !device_memory(scratch))
        return lfail(CSLBM_EINVAL, "fields, output and scratch must be device memory");
    const Box B = box_of(c, order);
    double* F = (double*)scratch;
    k_pad<<<dim3((unsigned)((B.Ne + TBL - 1) / TBL), (unsigned)ncomp), TBL, 0, c->stream>>>(B, f, order, F);
    k_grad<<<dim3((unsigned)((B.N + TBL - 1) / TBL), (unsigned)ncomp), TBL, 0, c->stream>>>(B, ncomp, F, out);
    c->launches += 2;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lfail(CSLBM_ECUDA, std::string("lattice gradient: ") + cudaGetErrorString(e));
    return CSLBM_OK;
}

}  // namespace lder
}  // namespace cslbm

using namespace cslbm::lder;

extern "C" {

cslbm_status cslbm_lattice_gradient_scratch_bytes(const cslbm_ctx* c, int ncomp, int order, size_t* bytes)
{
    if (!c || !bytes || ncomp < 1) return lfail(CSLBM_EINVAL, "bad argument");
    if (cslbm_status s = check_order(c, order)) return s;
    *bytes = pad_bytes(c, ncomp, order);
    return CSLBM_OK;
}

cslbm_status cslbm_lattice_gradient(cslbm_ctx* c, const double* f, int ncomp, int order, double* grad, void* scratch,
                                    size_t scratch_bytes)
{
    return gradient(c, f, ncomp, order, grad, scratch, scratch_bytes);
}

cslbm_status cslbm_metric_lattice_scratch_bytes(const cslbm_ctx* c, int order, size_t* bytes)
{
    if (!c || !bytes) return lfail(CSLBM_EINVAL, "bad argument");
    if (cslbm_status s = check_order(c, order)) return s;
    *bytes = 18 * (size_t)c->N * sizeof(double) + pad_bytes(c, 6, order);
    return CSLBM_OK;
}

cslbm_status cslbm_set_metric_lattice(cslbm_ctx* c, const double* g6, int order, void* scratch, size_t scratch_bytes)
{
    size_t need = 0;
    if (cslbm_status s = cslbm_metric_lattice_scratch_bytes(c, order, &need)) return s;
    if (!g6 || !scratch || scratch_bytes < need) return lfail(CSLBM_ENOMEM, "scratch smaller than required");
    double* dg = (double*)scratch;
    const size_t dg_bytes = 18 * (size_t)c->N * sizeof(double);
    if (cslbm_status s = gradient(c, g6, 6, order, dg, (char*)scratch + dg_bytes, scratch_bytes - dg_bytes)) return s;
    return cslbm_set_metric(c, g6, dg, 1);
}

cslbm_status cslbm_update_metric_lattice(cslbm_ctx* c, const double* g6, const double* Jnew9, int order, void* scratch,
                                         size_t scratch_bytes)
{
    size_t need = 0;
    if (cslbm_status s = cslbm_metric_lattice_scratch_bytes(c, order, &need)) return s;
    if (!g6 || !Jnew9 || !scratch || scratch_bytes < need) return lfail(CSLBM_ENOMEM, "scratch smaller than required");
    if (!device_memory(Jnew9)) return lfail(CSLBM_EINVAL, "Jnew9 must be device memory");
    double* dg = (double*)scratch;
    const size_t dg_bytes = 18 * (size_t)c->N * sizeof(double);
    if (cslbm_status s = gradient(c, g6, 6, order, dg, (char*)scratch + dg_bytes, scratch_bytes - dg_bytes)) return s;
    return cslbm_update_metric(c, g6, dg, Jnew9, 1);
}

}  // extern "C"
