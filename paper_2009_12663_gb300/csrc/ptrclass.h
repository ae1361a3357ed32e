/*
 * Where a caller's array lives, decided from its CUDA pointer attributes.
 * Plain C with no CUDA types, so the decision can be compiled and checked on
 * a machine without a GPU.
 *
 * Every entry point takes arrays that may be host or device memory.  A
 * device array must belong to the device that is current when the call is
 * made: the kernels run there, and a pointer into another GPU's memory
 * (without peer access set up by the caller) would fault instead of
 * returning an error.  Managed memory can be reached from any device.
 */
#ifndef GBFWI_PTRCLASS_H
#define GBFWI_PTRCLASS_H

/* the values of cudaMemoryType (checked against the runtime's enum where the
 * runtime header is available) */
#define GB_MEMTYPE_UNREGISTERED 0
#define GB_MEMTYPE_HOST 1
#define GB_MEMTYPE_DEVICE 2
#define GB_MEMTYPE_MANAGED 3

#define GB_PTR_HOST 0      /* pageable or pinned host memory: staged by the library */
#define GB_PTR_LOCAL 1     /* memory of the current device (or managed memory) */
#define GB_PTR_FOREIGN 2   /* memory of another device: rejected with GBFWI_EINVAL */

static inline int gb_classify_pointer(int memtype, int ptr_device, int current_device)
{
    if (memtype == GB_MEMTYPE_DEVICE) return ptr_device == current_device ? GB_PTR_LOCAL : GB_PTR_FOREIGN;
    if (memtype == GB_MEMTYPE_MANAGED) return GB_PTR_LOCAL;
    return GB_PTR_HOST;
}

#endif
