"""GB300-native track-repeating proton dose engine (placeholder, filled in below)."""
