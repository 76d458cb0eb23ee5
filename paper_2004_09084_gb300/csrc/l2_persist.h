// Bookkeeping for the persisting part of L2 that the frame kernel's
// access-policy window takes.  A windowed decode raises the context's
// persisting-L2 limit (cudaLimitPersistingL2CacheSize) to its window size, and
// the part set aside stays lost to every later kernel in the context while the
// limit stands (measured on GB300: grouped decodes of 128 frames ran 26 %
// slower with 68 MB set aside than with the default 25 MB, and as fast as
// before once the limit was put back).  The library notes each windowed decode
// and, before its next launch without a window on that device, resets the
// persisting lines and puts the limit back to the value it found.
#pragma once

#include <cstddef>

namespace qcmet {

// A decode under a persisting window is being issued on the current device.
// raised: the library raised the persisting-L2 limit for it, from prior_limit.
// Only the first raise since the last release records its prior value.
void note_persisting_l2(bool raised, size_t prior_limit);

// If a windowed decode was issued on the current device since the last
// release: reset the context's persisting L2 lines to normal and put the
// persisting-L2 limit back to the value recorded by the first raise.  Both are
// host calls that act when they return, not in stream order: a windowed kernel
// still running then keeps less of its state in L2 (its speed changes, not its
// results).  A failure of either is cleared and ignored; it can affect only the
// speed of later kernels.
void release_persisting_l2();

}  // namespace qcmet
