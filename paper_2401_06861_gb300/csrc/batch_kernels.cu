// Batched parameter-set evaluation (filled in below).
#include <cuda_runtime.h>
