"""GB300-native MegaParticles hot path (CUDA kernels behind a C ABI)."""
