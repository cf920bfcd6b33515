// Instantiates the reconstruction kernels for one thread count (VC_NT, set by the build).
#include "decode_kernels.cuh"

#ifndef VC_NT
#error "VC_NT must be defined (256, 512 or 1024)"
#endif

namespace vc {
namespace {

template <int L, typename GT, bool RANS>
void* kernel_for(bool batched) {
  if constexpr (L >= 6) {
    (void)batched;  // one kernel for every schedule
    return reinterpret_cast<void*>(&dev::decode_scratch_kernel<L, GT, RANS, VC_NT>);
  } else {
    return batched ? reinterpret_cast<void*>(&dev::decode_batched_kernel<L, GT, RANS, VC_NT>)
                   : reinterpret_cast<void*>(&dev::decode_grid_kernel<L, GT, RANS, VC_NT>);
  }
}

}  // namespace

#define VC_CAT2(a, b) a##b
#define VC_CAT(a, b) VC_CAT2(a, b)
void* VC_CAT(pick_kernel_nt, VC_NT)(uint32_t L, bool gt16, bool rans, bool batched) {
#define VC_PICK(LL)                                                                          \
  case LL:                                                                                   \
    if (gt16) return rans ? kernel_for<LL, uint16_t, true>(batched) : kernel_for<LL, uint16_t, false>(batched); \
    return rans ? kernel_for<LL, uint8_t, true>(batched) : kernel_for<LL, uint8_t, false>(batched);
  switch (L) {
#if VC_NT == 256
    VC_PICK(1)
    VC_PICK(2)
    VC_PICK(3)
#endif
    VC_PICK(4)
    VC_PICK(5)
    VC_PICK(6)
    default:
      return nullptr;
  }
#undef VC_PICK
}

}  // namespace vc
