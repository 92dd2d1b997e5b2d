"""GB300-native Monte Carlo engine for the IC and LT diffusion models."""
