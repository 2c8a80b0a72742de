// Shared declarations of the batched multi-RHS low-precision apply
// (batched.cu, near_tc.cu, bsolve.cu): the per-mesh descriptor table and
// the near-panel work items.
#pragma once

#include "device_common.cuh"

namespace vfd {

constexpr int RT = 64;   // RHS per tile

// one operator of a batch, as the kernels see it (device-resident table)
struct MrMesh {
    int N, fl, k, kp, L, lmin, nlev, nleaf, nnode, has_near, has_far;
    long long xoff;   // first row of this mesh in the batch vectors
    const int *kb, *ke, *pw, *gcol, *goff, *rowptr, *colidx, *fptr, *fcol;
    const int64_t *poff;
    const void *D;            // near panels (FP32 rounded to TF32, or BF16)
    const void *Ulf, *S;      // flattened bases N x mt (every far level, rank padded), coupling nfar x kp x kp
    int mt;                   // nlev * kp
    const float *val;         // B + M in FP32 (CSR)
    const float *diag;        // diagonal of A in FP32 (compensated), B + M off it folded into D
    float *xhat, *yhat;       // far-field workspaces of this mesh: nnode x kp x R
    float *part;              // leaf projections of every level, nleaf x mt x R
};

// one (mesh, leaf) work item of the near-panel kernel, everything it needs in one load
struct NearItem {
    const void *D;       // the leaf's panel (row stride W)
    const int *gcol;     // the panel's gather columns (mesh-local DoFs, -1 = padding)
    int row0;            // first row of the leaf in the batch vectors
    int na, W;           // leaf rows, panel width (multiple of 8)
    int xoff;            // first row of the mesh in the batch vectors
    int mesh, pad;
};

}  // namespace vfd
