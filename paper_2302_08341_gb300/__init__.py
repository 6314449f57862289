"""GB300-native ensemble local-inertial flood model with an on-device
particle filter (arXiv 2302.08341).  The compute path is the CUDA library
``libflood.so`` behind the C ABI declared in ``include/flood.h``; this
package holds its ctypes binding and the seeded input generators."""
