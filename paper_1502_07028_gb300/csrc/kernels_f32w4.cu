// FP32 reduction (PTCA_MIXED) in 4-warp CTAs -- one warp group per matrix --
// for matrix orders up to 128: more resident matrices per SM than the 8-warp
// kernels (three against two at n = 128).  Sweep kernels only.
#define PTCA_T float
#define PTCA_SYM(x) x##_f32w4
#define PTCA_NT_LIST(X) X(1) X(2) X(4)
#define PTCA_NWP 4
#define PTCA_AUX 0
#include "kernels_prec.inc"
