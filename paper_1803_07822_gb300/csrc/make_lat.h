// The device-side lattice description of a context (host code).
#pragma once

#include "ctx.h"
#include "lbm_device.cuh"

namespace cslbm {

inline Lat make_lat(const cslbm_ctx* c)
{
    Lat L;
    for (int a = 0; a < 3; a++) {
        L.n[a] = c->n[a];
        L.bclo[a] = c->p.bc_lo[a];
        L.bchi[a] = c->p.bc_hi[a];
        L.fext[a] = c->p.fext[a];
    }
    L.N = c->N;
    L.omega = 1.0 / c->p.tau;
    L.kvisc = 1.0 - 0.5 / c->p.tau;
    L.theta = c->theta;
    for (int k = 0; k < 6; k++) L.face[k] = c->face[k];
    return L;
}

}  // namespace cslbm
