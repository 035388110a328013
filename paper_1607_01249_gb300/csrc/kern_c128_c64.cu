// kern_c128_c64.cu -- kernel instantiations for one dtype pair (see kernels_pair.cuh).
#define TTC_DIN ttc::DT_C128
#define TTC_DOUT ttc::DT_C64
#define TTC_PAIR c128_c64
#include "kernels_pair.cuh"
