#include "internal.h"
#include "dd.h"
namespace gc { void dd_release() {} }
extern "C" int gc_calibrate_dd_cohjones(const void*, const void*, const gc_layout*, void*, const gc_options*, int32_t*, double*, int32_t*, void*) { return GC_ERR_DTYPE; }
