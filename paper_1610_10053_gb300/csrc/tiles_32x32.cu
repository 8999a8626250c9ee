// Fused 2-D kernels and preconditioner with 32 x 32 tiles (see tiles.h).
#include "tiles_impl.cuh"

template int fused2d_apply_t<32, 32>(music_grid *, int, const double *, const double *, const void *, int, void *,
                                   int, double *, double, double, cudaStream_t);
template int precond2d_apply_t<32, 32>(music_grid *, double, const void *, void *, int, cudaStream_t);
