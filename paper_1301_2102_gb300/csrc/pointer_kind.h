// Classification of a caller's pointer from its cudaPointerAttributes, as a plain host function of
// the attribute values (no CUDA types), so that it can be checked without a GPU.
#pragma once

namespace bmr {

enum class MemKind { host, device, other_device };

// attributes_ok: cudaPointerGetAttributes succeeded; type: cudaMemoryType (0 unregistered, 1 host,
// 2 device, 3 managed); ptr_device: the attributes' device; current_device: cudaGetDevice.
// Device memory of another GPU is `other_device`: the kernels of this library must not touch it
// (without peer access that is an illegal address).
inline MemKind mem_kind(bool attributes_ok, int type, int ptr_device, int current_device) {
  if (!attributes_ok) return MemKind::host;
  if (type == 3) return MemKind::device;
  if (type != 2) return MemKind::host;
  return (current_device >= 0 && ptr_device == current_device) ? MemKind::device : MemKind::other_device;
}

}  // namespace bmr
