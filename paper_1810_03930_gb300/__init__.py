"""GB300 (sm_103a) PLAM / PCAL hot path: Python binding of the C ABI in include/plam.h."""
