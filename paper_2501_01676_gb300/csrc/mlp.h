// Internal interface of the learned edge-GEP skip (features + MLP).
#pragma once
#include <cuda_runtime.h>

#include "../../include/bddc.h"

struct EdgeDesc {
    int axis;          // direction of the edge line
    int lo, hi;        // node index range of the interior dofs along the axis
    int c0, c1;        // node coordinates in the two other directions (increasing axis order)
    int subs[4];       // subdomains sharing the edge (-1 padded)
    int m;             // largest slab element count over the subdomains
    double theta;      // Theta_E of the edge GEP
};

int mlp_edge_features(const EdgeDesc* ed, int nedges, const double* nu, const double* beta, const double bconst[3],
                      const int* sx, const int* sy, const int* sz, int nsx, int nsy, int Ex, int Ey,
                      const double h[3], float* F, cudaStream_t st);
int mlp_probs(const float* params_dev, const float* X, int rows, float* P, cudaStream_t st);
