"""GB300-native split-operator propagator for the time-dependent Schroedinger equation
(arXiv:1306.3247). The compute path is the CUDA library built from csrc/ behind the
C ABI in include/wavepacket_gpu.h; `wavepacket` is its Python binding and
`workloads` holds the seeded synthetic inputs."""
