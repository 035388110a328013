// kern_f32_e4m3.cu -- kernel instantiations for one dtype pair (see kernels_pair.cuh).
#define TTC_DIN ttc::DT_F32
#define TTC_DOUT ttc::DT_E4M3
#define TTC_PAIR f32_e4m3
#include "kernels_pair.cuh"
