// Interpreter variant: complex64 bulk with FP64 state, one thread-block cluster per instance.
#include "ttn_variant.cuh"

int ttn_variant_mix_clu(const TtnVariantArgs& a) { return variant_launch<double2, float2, Clu>(a); }
int ttn_variant_mix_clu_init() { return variant_init<double2, float2, Clu>(); }
int ttn_variant_mix_clu_capacity(int cluster, int* max_active) { return variant_capacity<double2, float2>(cluster, max_active); }
