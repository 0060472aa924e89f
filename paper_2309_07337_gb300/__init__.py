"""GB300-native persistent neighbourhood all-to-all-v (placeholder; binding follows)."""
