"""GB300-native moving-PML sweeping preconditioner (placeholder, filled below)."""
