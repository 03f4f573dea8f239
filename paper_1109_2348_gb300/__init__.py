"""GB300-native forward Burrows-Wheeler block sort (placeholder; binding added below)."""
