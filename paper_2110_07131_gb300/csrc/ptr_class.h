// Where a caller's buffer lives relative to the GPU an index is on.
//
// The entry points accept host or device buffers and tell them apart with
// cudaPointerGetAttributes.  Device memory of ANOTHER GPU must be refused
// (RMIPS_ERR_ARG): the kernels run on the index's GPU and would otherwise
// read or write memory they cannot reach.  This header holds only the
// decision, on the attribute values, so that it can be checked on a machine
// without a GPU.  `type` is a cudaMemoryType value: 0 unregistered host,
// 1 pinned host, 2 device, 3 managed (unified) memory.
#pragma once

namespace rmips {

enum : int { PTR_HOST = 0, PTR_DEVICE = 1, PTR_OTHER_DEVICE = 2 };

inline int ptr_class_of(int type, int ptr_device, int index_device) {
  if (type == 3) return PTR_DEVICE;                 // managed: reachable from every GPU
  if (type == 2) return ptr_device == index_device ? PTR_DEVICE : PTR_OTHER_DEVICE;
  return PTR_HOST;                                  // pageable or pinned host memory
}

}  // namespace rmips
