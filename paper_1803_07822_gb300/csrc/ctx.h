// Internal context of the library (host side), shared by the C ABI and the
// per-storage-format kernel units.  Not part of the public interface.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "../../include/cslbm.h"
#include "rows_plan.h"

struct cslbm_ops;

// Resources of the row-staged step pass, made at creation when it applies:
// its plan and the tensor maps of the buffers it stages (populations,
// geometry and history per ping-pong buffer, rho u).
struct cslbm_rows {
    int ok;        // the row pass applies (plan and maps made)
    int fused_ok;  // ... and the fused form (non-periodic axis 2, cooperative launch, smem)
    cslbm::rows::Plan plan;
    CUtensorMap pop[2];   // [19][n2][n1][n0] populations, box n0 x TR
    CUtensorMap pop3[2];  // the same, box n0 x TR x 1 x 3 (three planes that pull from one row)
    CUtensorMap jf;       // rho u as [4 N / JL][JL] floats, box JL x JR (the TR + 2 rows of a layer)
    CUtensorMap jf3;      // rho u as [n2][4 n0 n1 / JL][JL] floats, box JL x JR x 3 (three layers)
    CUtensorMap geo[2];   // [25][N] geometry, box NT x 25
    CUtensorMap hist[2];  // [10][N] history, box NT x 10
    CUtensorMap geo1[2];  // sqrt(g) alone, box NT x 1
    CUtensorMap hist4[2]; // A and B of the history, box NT x 4
    unsigned* done;       // [iterations] CTAs that published each momentum iteration (cumulative)
    unsigned epoch;       // fused launches so far
    unsigned long long test_wait_ns;  // next fused launch only: wait limit (0: the default)
    int test_withhold;    // next fused launch only: iteration CTA 0 does not count as published (-1: none)
    unsigned off_m, off_sg, off_h4, off_js, fused_bytes;
};

struct cslbm_ctx {
    cslbm_params p;
    int n[3];
    long long N;
    double theta;
    cudaStream_t stream;
    int device;
    int n_sm;        // multiprocessors of the device
    size_t s_bytes;  // bytes of one stored population
    size_t r_bytes;  // bytes of one compute-precision value
    void* P[2];      // [19][N] stored populations (pull layout, weight shifted)
    void* H[2];      // [10][N] forcing-history coefficients
    void* G[2];      // [25][N] geometry: sqrt(g), g^ij, Gamma
    void* J;         // [9][N] current chart Jacobian at the precision R of the arithmetic (FP64 for FP64
                     // storage, FP32 otherwise)
    void* jf;        // [N] rho u (x, y, z, unused) of every node
    double* face[6]; // [3][face nodes] boundary velocity of non-periodic faces
    long long face_n[6];
    double* scratch; // 64 doubles of reduction space
    double* staging; // host-transfer staging, chunk * 24 doubles
    long long chunk; // nodes per staging chunk
    int pc, hc, gc;  // current buffer of P, H, G
    int has_state;
    int metric_check_pending;  // a metric kernel ran without a host check
    const cslbm_ops* ops;
    // profiling
    cslbm_rows rows;
    struct {
        void* ws;  // adjoint fields (cslbm_adjoint_attach), or null
        int lp;    // which of the two adjoint buffers holds the current adjoint state
    } adj;
    int prof;
    std::vector<cudaEvent_t> ev;  // start/stop pairs of profiled steps
    long long prof_steps;
    long long launches;
};

// Per-storage-format entry points (one kernel unit per format).
// Node ranges: a launch touches nodes [v0, v0 + cnt); FP64 inputs given as
// [components][stride] with the node's entry at (v - v0).
struct cslbm_ops {
    // geometry of G[dst] from g6/dg18; *bad set non-zero on det g <= 0
    void (*metric)(const cslbm_ctx*, const double* g6, const double* dg18, long long stride,
                   long long v0, long long cnt, int dst, int* bad);
    // P[pc] slots of f^eq(rho,u) (history still zero)
    void (*init_scatter)(const cslbm_ctx*, const double* rho, const double* u3, long long stride,
                         long long v0, long long cnt);
    // jf <- rho u of the current state
    void (*momentum_field)(const cslbm_ctx*);
    // one time step P[pc],H[hc] -> P[1-pc],H[1-hc] (momentum pass + step
    // pass); force_only: only H[1-hc] from the momentum field jf.  Returns
    // the number of kernels it launched.
    int (*step)(cslbm_ctx*, int force_only);
    // P[pc] slots -= F/2 of H[hc] (end of initialisation)
    void (*half_shift)(const cslbm_ctx*);
    // chart change for nodes [v0, v0+cnt): P[pc],H[hc],G[gc] -> P[1-pc],H[1-hc] with G[1-gc]
    void (*transform)(const cslbm_ctx*, const double* Jnew, long long stride, long long v0,
                      long long cnt);
    // the whole node-wise chart change in one pass (device inputs of every
    // node): G[1-gc] from g6/dg18, then P[pc],H[hc] -> P[1-pc],H[1-hc] and J
    // replaced by Jnew; *bad set non-zero on det g <= 0
    void (*chart_change)(const cslbm_ctx*, const double* g6, const double* dg18, const double* Jnew, int* bad);
    void (*chart_change_mixed)(const cslbm_ctx*, const double* g6, const float* dg18, const float* Jnew, int* bad);
    // chart change with interpolation: the transformation inputs of every node
    // into scratch [20][N] (precision R), then every node of P[1-pc],H[1-hc]
    // from them at psi3 [3][N] (old lattice coordinates) with G[1-gc]; J (old)
    // is read, not written
    void (*transform_interp)(const cslbm_ctx*, const double* Jnew, const double* psi3, void* scratch);
    // rho, u (or v) of nodes [v0, v0+cnt) into out arrays with the given stride
    void (*readout)(const cslbm_ctx*, double* rho, double* u3, long long stride, long long v0,
                    long long cnt, int cartesian);
    // scratch[0] += sum sqrt(g) rho
    void (*mass)(const cslbm_ctx*, double* acc);
    // acc[0..2] += wall force of face (axis, side)
    void (*wall_force)(const cslbm_ctx*, int axis, int side, double* acc);
    // acc[0] += number of unstable nodes
    void (*check)(const cslbm_ctx*, double* acc);
};

// flag the row-staged step pass sets when one of its bounded waits runs out
// (an int in the reduction scratch, zero from creation; cslbm_check reads it)
inline int* step_error_flag(const cslbm_ctx* c) { return (int*)(c->scratch + 40); }

// records the message cslbm_last_error() returns on this thread; returns s
cslbm_status cslbm_record_error(cslbm_status s, const char* msg);

extern const cslbm_ops cslbm_ops_fp32;
extern const cslbm_ops cslbm_ops_fp16;
extern const cslbm_ops cslbm_ops_bf16;
extern const cslbm_ops cslbm_ops_fp64;
