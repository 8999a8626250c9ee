// The persistent batched kernel with 32 x 16 tiles, FP32 Krylov type (one translation unit
// per shape and precision, so the library builds in parallel).
#include "batched_impl.cuh"

namespace batch {
MUSIC_BATCHED_INSTANTIATE_F32(32, 16)
}
