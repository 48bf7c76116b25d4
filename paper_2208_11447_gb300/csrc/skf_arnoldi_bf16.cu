// Reduced-precision truncated Arnoldi, BF16 basis storage (instantiation of
// the kernels in skf_arnoldi_lp.cuh).
#include "skf_arnoldi_lp.cuh"

namespace skf {

skf_status arnoldi_run_bf16(const skf_csr *A, const skf_sketch *S, const double *b, int m, int k, void *V,
                            int64_t ldv, double *vscale, double *SV, double *SAV, double *H, int *iscal,
                            skf_info *info, cudaStream_t st, const StepHook *hook, int vring) {
    return lp::arnoldi_run_lp<__nv_bfloat16>(A, S, b, m, k, (__nv_bfloat16 *)V, ldv, vscale, SV, SAV, H, iscal,
                                             info, st, hook, vring);
}

}  // namespace skf
