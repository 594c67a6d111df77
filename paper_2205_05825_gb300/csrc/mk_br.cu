// Blind-rotation instantiation for one (ring dimension, field, variant),
// chosen by the build with -DMK_LOGN=<log2 N> -DMK_FIELD=<0|1>
// -DMK_VARIANT=<v>; field 0 = Goldilocks (MK_FORM_NTT), 1 = two 28-bit primes
// (MK_FORM_NTT2), 2 = FP64 FFT (MK_FORM_FFT, one variant); the variant table
// is in mk_internal.h.
#include "mk_bootstrap.cuh"
#include "mk_bootstrap_fft.cuh"
#include "mk_bootstrap_split.cuh"
#include "mk_netlist.cuh"
#include "mk_bootstrap_staged.cuh"

#ifndef MK_LOGN
#error "compile with -DMK_LOGN=<log2 N> -DMK_VARIANT=<v>"
#endif

#define MK_CAT2(a, b, c, d, e, f) a##b##c##d##e##f
#define MK_CAT(a, b, c, d, e, f) MK_CAT2(a, b, c, d, e, f)
#define MK_FN MK_CAT(launch_bootstrap_logn, MK_LOGN, _f, MK_FIELD, _v, MK_VARIANT)

namespace mk {
cudaError_t MK_FN(const LaunchShape &S, const DeviceKeys &K, const GateDesc *desc, const uint32_t *ct_a,
                  const uint32_t *ct_b, const uint32_t *abar_in, int64_t max_steps, uint32_t *ext,
                  uint32_t *acc_out, uint32_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    constexpr int NPF = kVariantNpf[MK_VARIANT];
    constexpr int MINB = kVariantMinBlocks[MK_VARIANT];
    constexpr bool TWG = kVariantTwg[MK_VARIANT] != 0;
    constexpr int EPT = kVariantEpt[MK_VARIANT];
#if MK_FIELD == 2
    (void)NPF;
    (void)MINB;
    (void)TWG;
    (void)EPT;
    return br::launch_bootstrap_fft<MK_LOGN - 1>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out, count,
                                                 st);
#else
#if MK_FIELD == 0
    using F = br::FieldGold;
#else
    using F = br::FieldDual;
#endif
    if constexpr (kVariantKind[MK_VARIANT] == 1) {
        (void)MINB;
        (void)TWG;
        (void)EPT;
        return br::launch_staged<F, MK_LOGN, NPF>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out, count,
                                                  st);
    } else if constexpr (kVariantKind[MK_VARIANT] == 2 && MK_FIELD == 1) {
        (void)TWG;
        (void)EPT;
        return br::launch_split<MK_LOGN, NPF, MINB>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out, count,
                                                    st);
    } else if constexpr (kVariantKind[MK_VARIANT] == 2) {  // no split form of the one-prime field: variant 2's kernel
        (void)NPF;
        (void)MINB;
        (void)TWG;
        (void)EPT;
        return br::launch_bootstrap<F, MK_LOGN, kVariantNpf[2], kVariantMinBlocks[2], kVariantTwg[2] != 0,
                                    kVariantEpt[2]>(S, K, desc, ct_a, ct_b, abar_in, max_steps, ext, acc_out, count,
                                                    st);
    } else {
        return br::launch_bootstrap<F, MK_LOGN, NPF, MINB, TWG, EPT>(S, K, desc, ct_a, ct_b, abar_in, max_steps,
                                                                     ext, acc_out, count, st);
    }
#endif
}
}  // namespace mk

#if MK_VARIANT == 2 && MK_FIELD != 2
// The persistent netlist kernel of this (ring dimension, field), with variant
// 2's blind-rotation parameters.
#define MK_NL_FN MK_CAT(launch_netlist_logn, MK_LOGN, _f, MK_FIELD, , )
namespace mk {
cudaError_t MK_NL_FN(const LaunchShape &S, const DeviceKeys &K, const NetlistArgs &A, uint32_t sm_count,
                     cudaStream_t st) {
#if MK_FIELD == 0
    using F = br::FieldGold;
#else
    using F = br::FieldDual;
#endif
    return br::launch_netlist<F, MK_LOGN, kVariantNpf[2], kVariantMinBlocks[2], kVariantTwg[2] != 0, kVariantEpt[2]>(
        S, K, A, sm_count, st);
}
}  // namespace mk
#endif
