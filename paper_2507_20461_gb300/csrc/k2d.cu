/* Stage kernels of the 2D compact GKS with GENO reconstruction (FP64 and mixed precision). */
#include "launch.cuh"

namespace gks {
GKS_INSTANTIATE(2)
}
