// Definitions of the launchers declared in launch.h, included by the
// per-type translation units (the type's kernels are instantiated there).
#include "kernels.cuh"
#include "launch.h"

namespace sp {

#define SP_PICK(FN, T, ADJV, BIGV, ...)                                         \
  do {                                                                          \
    if (ADJV) {                                                                 \
      if (BIGV) FN<T, true, true><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);   \
      else FN<T, true, false><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);       \
    } else {                                                                    \
      if (BIGV) FN<T, false, true><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);  \
      else FN<T, false, false><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);      \
    }                                                                           \
  } while (0)

// forward-only types (the double-float form has no adjoint) instantiate ADJ = false only
#define SP_PICK_FWD(FN, T, BIGV, ...)                                           \
  do {                                                                          \
    if (BIGV) FN<T, false, true><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);    \
    else FN<T, false, false><<<l.grid, l.threads, l.smem, l.stream>>>(__VA_ARGS__);        \
  } while (0)

}  // namespace sp
