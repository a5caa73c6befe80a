// credit_kernels.cu -- instantiates the row kernels for one input dtype.
//
// The build compiles this file three times with -DCREDIT_TIN=0 (FP32),
// 1 (BF16) and 2 (FP8-E4M3) so that the three object files compile in
// parallel.  Each exports credit::kernels_tin<N>(op, out_dtype, &set), which
// fills the kernel table the host dispatcher launches from.
#include "credit_ring_tm.cuh"

#ifndef CREDIT_TIN
#error "CREDIT_TIN must be defined (0 = FP32, 1 = BF16, 2 = FP8-E4M3)"
#endif

#define CREDIT_CAT2(a, b) a##b
#define CREDIT_CAT(a, b) CREDIT_CAT2(a, b)

namespace credit {

template <int OP, int TIN, int TOUT>
static void fill_set(KernelSet *ks) {
    ks->ring = reinterpret_cast<const void *>(&k_ring<OP, TIN, TOUT>);
    ks->ring_tm = nullptr;
    if constexpr (OP != OP_LSE && !(TOUT == DT_E4M3 && (OP == OP_LN || OP == OP_RMS)))
        ks->ring_tm = reinterpret_cast<const void *>(&k_ring_tm<OP, TIN, TOUT>);
    ks->tp_fused = reinterpret_cast<const void *>(&k_tp_fused<OP, TIN, TOUT>);
    ks->tp_stats = reinterpret_cast<const void *>(&k_tp_stats<OP, TIN>);
    ks->tp_amax = nullptr;
    ks->tp_apply = nullptr;
    ks->tp_lse_final = nullptr;
    if constexpr (OP == OP_LN || OP == OP_RMS) {
        if constexpr (TOUT == DT_E4M3) ks->tp_amax = reinterpret_cast<const void *>(&k_tp_amax<OP, TIN>);
    }
    if constexpr (OP == OP_LSE) ks->tp_lse_final = reinterpret_cast<const void *>(&k_tp_lse_final<TIN>);
    else ks->tp_apply = reinterpret_cast<const void *>(&k_tp_apply<OP, TIN, TOUT>);
}

template <int OP, int TIN>
static bool fill_out(int tout, KernelSet *ks) {
    if constexpr (OP == OP_LSE) {
        if (tout != DT_F32) return false;
        fill_set<OP, TIN, DT_F32>(ks);
        return true;
    } else if constexpr (OP == OP_Q8) {  // FP32 / BF16 rows -> int8 codes
        if (tout != DT_I8 || TIN == DT_E4M3) return false;
        fill_set<OP, TIN, DT_I8>(ks);
        return true;
    } else {
        switch (tout) {
        case DT_F32: fill_set<OP, TIN, DT_F32>(ks); return true;
        case DT_BF16: fill_set<OP, TIN, DT_BF16>(ks); return true;
        case DT_E4M3: fill_set<OP, TIN, DT_E4M3>(ks); return true;
        default: return false;
        }
    }
}

bool CREDIT_CAT(kernels_tin, CREDIT_TIN)(int op, int tout, KernelSet *ks) {
    switch (op) {
    case OP_SOFTMAX: return fill_out<OP_SOFTMAX, CREDIT_TIN>(tout, ks);
    case OP_LSE: return fill_out<OP_LSE, CREDIT_TIN>(tout, ks);
    case OP_LN: return fill_out<OP_LN, CREDIT_TIN>(tout, ks);
    case OP_RMS: return fill_out<OP_RMS, CREDIT_TIN>(tout, ks);
    case OP_Q8: return fill_out<OP_Q8, CREDIT_TIN>(tout, ks);
    default: return false;
    }
}

}  // namespace credit
