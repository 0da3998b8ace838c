// FP32 reduction (PTCA_MIXED): NT = 1, 2, 4, 7 -> matrix orders up to 224.
#define PTCA_T float
#define PTCA_SYM(x) x##_f32
#define PTCA_NT_LIST(X) X(1) X(2) X(4) X(7)
#include "kernels_prec.inc"
