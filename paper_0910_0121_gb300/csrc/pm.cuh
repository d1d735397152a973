// PM plan and driver shared by pm.cu and api.cu (internal).
#pragma once
#include <cufft.h>

#include "common.cuh"

namespace greem {
struct PmPlan {
    int n = 0;
    cufftHandle r2c = 0, c2r = 0;
    bool have = false;
};
int pm_plan(PmPlan &pl, int n, cudaStream_t s);
void pm_plan_destroy(PmPlan &pl);
int run_pm(const PmPlan &pl, const double *pos, const double *xs, const double *ys, const double *zs,
           const float *mass, const uint32_t *perm, uint32_t N, double L, int n, int scheme, int pow2_e,
           const float *table, float *grid, cufftComplex *spec, cufftComplex *tmp, float *acc, int accumulate,
           cudaStream_t s, int nsm);
}  // namespace greem
