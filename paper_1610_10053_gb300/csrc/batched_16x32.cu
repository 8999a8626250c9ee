// The persistent batched kernel with 16x32 tiles (one translation unit per
// shape, so the library builds in parallel).
#include "batched_impl.cuh"

namespace batch {
MUSIC_BATCHED_INSTANTIATE(16, 32)
}
