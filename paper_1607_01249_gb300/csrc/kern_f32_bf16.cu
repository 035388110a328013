// kern_f32_bf16.cu -- kernel instantiations for one dtype pair (see kernels_pair.cuh).
#define TTC_DIN ttc::DT_F32
#define TTC_DOUT ttc::DT_BF16
#define TTC_PAIR f32_bf16
#include "kernels_pair.cuh"
