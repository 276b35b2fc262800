"""GB300-native path-integral Monte Carlo data assimilation (Quinn & Abarbanel)."""
