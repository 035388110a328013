// kern_f64_f32.cu -- kernel instantiations for one dtype pair (see kernels_pair.cuh).
#define TTC_DIN ttc::DT_F64
#define TTC_DOUT ttc::DT_F32
#define TTC_PAIR f64_f32
#include "kernels_pair.cuh"
