"""GB300-native multi-scale low rank decomposition (Ong & Lustig)."""
