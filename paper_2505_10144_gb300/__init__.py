"""GB300-native (sm_103a) foveated, popping-free Gaussian-splat rasterizer (VRSplat hot path)."""
