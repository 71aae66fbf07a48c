// k_split_low.cu -- the 2..5-slice instantiations of the split-BF16 tensor-core path: the same
// sources as k_split.cu compiled as a second translation unit, so that the build compiles the two
// halves of the row-kernel instantiations in parallel.
#define NPF_SPLIT_LOW 1
#include "k_split.cu"
