// Reduced-precision truncated Arnoldi, FP32 basis storage (instantiation of
// the kernels in skf_arnoldi_lp.cuh).
#include "skf_arnoldi_lp.cuh"

namespace skf {

skf_status arnoldi_run_f32(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, float *V,
                           int64_t ldv, double *vscale, double *SV, double *SAV, double *H, int *iscal,
                           skf_info *info, cudaStream_t st, const StepHook *hook, int vring) {
    return lp::arnoldi_run_lp<float>(A, S, b, m, k, V, ldv, vscale, SV, SAV, H, iscal, info, st, hook, vring);
}

skf_status arnoldi_run_f32_block(const skf_csr *A, const skf_sketch *S, int nr, const double *const *b, int m, int k,
                                 float *const *V, int64_t ldv, double *const *vscale, double *const *SV,
                                 double *const *SAV, double *const *H, int *const *iscal, skf_info *const *info,
                                 cudaStream_t st) {
    return lp::arnoldi_run_lp_block<float>(A, S, nr, b, m, k, V, ldv, vscale, SV, SAV, H, iscal, info, st);
}

}  // namespace skf
