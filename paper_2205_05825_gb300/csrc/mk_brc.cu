// Cluster (latency) blind-rotation instantiation for one (ring dimension,
// field), chosen by the build with -DMK_LOGN=<log2 N> -DMK_FIELD=<0|1>;
// field 0 = Goldilocks (MK_FORM_NTT), 1 = two 28-bit primes (MK_FORM_NTT2).
#include "mk_bootstrap_cluster.cuh"

#ifndef MK_LOGN
#error "compile with -DMK_LOGN=<log2 N> -DMK_FIELD=<0|1>"
#endif

#define MK_CCAT2(a, b, c, d) a##b##c##d
#define MK_CCAT(a, b, c, d) MK_CCAT2(a, b, c, d)
#define MK_CFN MK_CCAT(launch_cluster_logn, MK_LOGN, _f, MK_FIELD)
#define MK_CAPFN MK_CCAT(cluster_capacity_logn, MK_LOGN, _f, MK_FIELD)

namespace mk {
cudaError_t MK_CFN(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc, const uint32_t *ct_a,
                   const uint32_t *ct_b, const uint32_t *abar_in, int64_t max_steps, uint32_t *ext,
                   uint32_t *acc_out, uint32_t count, cudaStream_t st) {
#if MK_FIELD == 0
    using F = br::FieldGold;
#else
    using F = br::FieldDual;
#endif
    return br::launch_bootstrap_cluster<F, MK_LOGN>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out, count,
                                                    st);
}

int MK_CAPFN(uint32_t k, uint32_t n) {
#if MK_FIELD == 0
    using F = br::FieldGold;
#else
    using F = br::FieldDual;
#endif
    return br::cluster_capacity<F, MK_LOGN>(k, n);
}
}  // namespace mk
