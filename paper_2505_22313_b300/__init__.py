"""B300-native DOE scalar-diffraction library (placeholder, filled in below)."""
