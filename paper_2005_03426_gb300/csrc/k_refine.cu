// k_refine.cu -- S6: Ogita-Aishima refinement of the mixed-precision eigenpairs.
#include "mmf_internal.h"

cudaError_t mmf_launch_refine(const MmfLaunch& L, const double2* coef, double2* X, double* E,
                              double2* R, double2* S, double2* HX, double* E2, int iters,
                              int* status) {
    (void)L; (void)coef; (void)X; (void)E; (void)R; (void)S; (void)HX; (void)E2; (void)iters;
    (void)status;
    return cudaErrorNotSupported;
}
