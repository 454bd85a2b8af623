"""B300-native VMAS world step (placeholder; filled in below)."""
