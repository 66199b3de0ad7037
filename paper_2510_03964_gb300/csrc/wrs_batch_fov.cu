// The foveating variants of the batched kernel (wrs_push_batch_foveated):
// every stream's frame is foveated on read from its rendered image and mip
// levels (Sec. 4.3's post-process) by the consumers, as wrs_push_foveated
// does for one stream; instantiated here, apart from the plain batches, so the
// two sets compile in parallel.
#include "wrs_batch_kernel.cuh"
#include "wrs_internal.h"

namespace {

template <int FILTER>
const void* fov_fn(int fam) {
  switch (fam) {
    case kFamF16K48: return reinterpret_cast<const void*>(&batch_kernel<1, kFamF16K48, FILTER>);
    case kFamF32K48: return reinterpret_cast<const void*>(&batch_kernel<1, kFamF32K48, FILTER>);
    default: return reinterpret_cast<const void*>(&batch_kernel<1, kFamAll, FILTER>);
  }
}

}  // namespace

const void* wrs_batch_fov_kernel(int fam, int filter) {
  return filter == WRS_FILTER_BILINEAR ? fov_fn<WRS_FILTER_BILINEAR>(fam)
                                       : fov_fn<WRS_FILTER_BOX>(fam);
}
