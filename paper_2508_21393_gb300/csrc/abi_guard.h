// Exceptions never cross the C ABI.  An entry point that allocates host
// memory (statement copies, descriptor tables, host-side verifier tables)
// runs its body between VL_ABI_TRY and VL_ABI_CATCH(value): std::bad_alloc,
// or anything else a standard-library call throws, becomes `value` (the
// entry point's error result) with a message for vl_last_error().
#pragma once
#include <new>

namespace vl {
void set_last_error(const char* msg);
}

#define VL_ABI_TRY try {
#define VL_ABI_CATCH(fail)                                  \
  }                                                         \
  catch (const std::bad_alloc&) {                           \
    vl::set_last_error("host memory allocation failed");    \
    return fail;                                            \
  }                                                         \
  catch (...) {                                             \
    vl::set_last_error("host-side exception in the library"); \
    return fail;                                            \
  }
