// Interpreter variant: complex128 bulk, one thread block per instance.
#include "ttn_variant.cuh"

int ttn_variant_f64_solo(const TtnVariantArgs& a) { return variant_launch<double2, double2, Solo<256>>(a); }
int ttn_variant_f64_solo_init() { return variant_init<double2, double2, Solo<256>>(); }
