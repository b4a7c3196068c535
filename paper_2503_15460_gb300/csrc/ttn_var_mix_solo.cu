// Interpreter variant: complex64 bulk with FP64 state, one thread block per instance.
#include "ttn_variant.cuh"

int ttn_variant_mix_solo(const TtnVariantArgs& a) { return variant_launch<double2, float2, Solo<256>>(a); }
int ttn_variant_mix_solo_init() { return variant_init<double2, float2, Solo<256>>(); }
