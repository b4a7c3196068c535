// Interpreter variant: complex64 bulk with FP64 state, one thread block per
// instance, with the tcgen05 mode product for dimensions the tuning assigns
// to tensor cores.
#define TTN_WITH_TC 1
#include "ttn_variant.cuh"

int ttn_variant_mix_solo_tc(const TtnVariantArgs& a) { return variant_launch<double2, float2, Solo<256>>(a); }
int ttn_variant_mix_solo_tc_init() { return variant_init<double2, float2, Solo<256>>(); }
