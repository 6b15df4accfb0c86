"""GB300-native spectral Poisson solver (periodic -Δu = f on the unit cube)."""
