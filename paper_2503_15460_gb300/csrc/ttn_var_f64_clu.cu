// Interpreter variant: complex128 bulk, one thread-block cluster per instance.
#include "ttn_variant.cuh"

int ttn_variant_f64_clu(const TtnVariantArgs& a) { return variant_launch<double2, double2, Clu>(a); }
int ttn_variant_f64_clu_init() { return variant_init<double2, double2, Clu>(); }
int ttn_variant_f64_clu_capacity(int cluster, int* max_active) { return variant_capacity<double2, double2>(cluster, max_active); }
