"""GB300-native colour-temperature decolorization (placeholder, filled in below)."""
