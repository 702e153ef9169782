"""GB300-native Radsort: the per-digit LSD round of "Parallel O(sqrt n)
Overhead LSD Radix Sort" (Clausecker & Schintke) as hand-written CUDA for
sm_103a behind a C ABI (include/radsort.h).  The Python side only marshals
arguments; every step of the sort runs in the CUDA library."""
