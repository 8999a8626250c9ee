// Fused 2-D preconditioner with 64 x 16 tiles (see tiles.h); the stencil has
// no tile of this shape.
#include "tiles_impl.cuh"

template int precond2d_apply_t<64, 16>(music_grid *, double, const void *, void *, int, cudaStream_t);
